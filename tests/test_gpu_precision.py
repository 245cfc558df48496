"""Precision split: FP32 trajectories (with FP64 tallies) against FP64.

For a single-mode material both precisions draw from the same random words
(the FP32 uniform keeps the top 23 bits), so a particle follows the same
history in both unless a rounding difference flips a wall-versus-relaxation
decision.  The tests bound how often that happens and check that the
results agree within their statistical errors; the measured fractions are
printed for the record.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def _pair(P, prob):
    a = P.simulate(W.with_run(prob, precision="fp64"), arrays=False, record_particles=True)
    b = P.simulate(W.with_run(prob, precision="fp32"), arrays=False, record_particles=True)
    return a, b


def test_slab_fp32_follows_fp64(P):
    prob = W.gray_slab(n_particles=1_000_000, n_bins=0)
    a, b = _pair(P, prob)
    ra, rb = a["particles_rec"], b["particles_rec"]
    fate_a = np.rint(ra["sign"] * ra["L_axis"])  # 1 = crossed, 0 = returned (exact in FP64)
    fate_b = np.rint(rb["sign"] * rb["L_axis"])
    differ = np.mean((fate_a != fate_b) | (ra["n_seg"] != rb["n_seg"]))
    print(f"\nslab: fraction of particles whose history differs FP32 vs FP64: {differ:.2e}")
    assert differ < 1e-3
    assert abs(a["psi"] - b["psi"]) < 3.0 * a["psi_se"]
    # the FP32 per-particle crossing is exact: s L_x / L stays 0 or 1
    assert np.max(np.abs(rb["sign"] * rb["L_axis"] - fate_b)) < 1e-5


def test_film_fp32_follows_fp64(P):
    prob = W.silicon_film(n_particles=500_000, thickness=1e-7, material=dict(W.GRAY_UNIT, tau=1e-10, v=1000.0),
                          dTdz=-1e6)
    a, b = _pair(P, prob)
    ra, rb = a["particles_rec"], b["particles_rec"]
    same = (ra["n_seg"] == rb["n_seg"]) & (ra["n_scat"] == rb["n_scat"]) & (ra["n_wall"] == rb["n_wall"])
    differ = 1.0 - np.mean(same)
    rel = np.abs(ra["L_axis"][same] - rb["L_axis"][same]) / (np.abs(ra["L_axis"][same]) + 1e-7)
    print(f"\nfilm: histories differing {differ:.2e}; median relative path-length difference "
          f"{np.median(rel):.2e}")
    assert differ < 1e-3
    assert np.median(rel) < 1e-5
    assert abs(a["kappa"] - b["kappa"]) < 3.0 * np.hypot(a["kappa_se"], b["kappa_se"])


def test_silicon_film_precisions_agree_statistically(P):
    prob = W.silicon_film(n_particles=20_000_000)
    a = P.simulate(W.with_run(prob, precision="fp64"), arrays=False)
    b = P.simulate(W.with_run(prob, precision="fp32"), arrays=False)
    z = abs(a["kappa"] - b["kappa"]) / np.hypot(a["kappa_se"], b["kappa_se"])
    print(f"\nsilicon film: kappa fp64 {a['kappa']:.4f} fp32 {b['kappa']:.4f} (z = {z:.2f}); "
          f"segments {a['segments']} vs {b['segments']}")
    assert z < 3.0
    assert abs(a["segments"] / b["segments"] - 1) < 1e-3


# ------------------------------------------------------------------------
# The error of every FP32 result against FP64 on the same random words.  For
# multi-mode materials both precisions pick modes from the same 32-bit words
# (alias tables), so a particle keeps its FP64 history until a rounding
# difference flips a decision; in pored cells (dispersing billiards) such
# flips grow with the number of pore reflections.  Each test prints the
# fraction of histories that differ and the relative error of the result, and
# checks the error against its statistical bound.
def _differ(ra, rb):
    same = (ra["n_seg"] == rb["n_seg"]) & (ra["fate"] == rb["fate"]) & (ra["n_scat"] == rb["n_scat"])
    return 1.0 - float(np.mean(same))


def test_pored_film_kappa_fp32_error(P):
    n = 2_000_000
    a, b = _pair(P, W.porous_film(n_particles=n))
    ra, rb = a["particles_rec"], b["particles_rec"]
    # paired per-particle differences of s L: their mean is the FP32 bias
    d = rb["sign"] * rb["L_axis"] - ra["sign"] * ra["L_axis"]
    bias = d.mean() / np.mean(ra["sign"] * ra["L_axis"])
    bias_se = d.std(ddof=1) / np.sqrt(n) / abs(np.mean(ra["sign"] * ra["L_axis"]))
    rel = b["kappa"] / a["kappa"] - 1.0
    print(f"\npored film kappa: FP32 {b['kappa']:.5f} FP64 {a['kappa']:.5f} rel. error {rel:+.2e} "
          f"(paired bias {bias:+.2e} +- {bias_se:.1e}); histories differing {_differ(ra, rb):.3f}")
    assert abs(bias) < 3.0 * bias_se + 1e-6
    # (the library's kappa and the records' sums differ only by summation order)
    from tests.tolerances import sum_order_rtol
    assert rel == pytest.approx(bias, abs=sum_order_rtol(b, "fp32") + sum_order_rtol(a, "fp64"))


@pytest.mark.parametrize("kind", ["pulse", "initial"])
def test_transient_grid_fp32_error(P, kind):
    from tests.test_gpu_parity import homogeneity_pvalues
    n = 1_000_000
    if kind == "pulse":
        prob = W.porous_pulse(n_particles=n, grid=(8, 24, 24), n_samples=40, sample_dt=25e-12, t_final=1e-9)
    else:
        prob = W.porous_initial(n_particles=n)
    a = P.simulate(W.with_run(prob, precision="fp64"), record_particles=True)
    b = P.simulate(W.with_run(prob, precision="fp32"), record_particles=True)
    ga, gb = a["grid"].astype(np.int64), b["grid"].astype(np.int64)
    ns = ga.shape[0]
    # total-variation distance of the two count distributions per sample
    tv = 0.5 * np.abs(ga - gb).reshape(ns, -1).sum(axis=1) / n
    moved = np.abs(ga - gb).sum() / max(np.abs(ga).sum(), 1)
    print(f"\n{kind} grid: histories differing {_differ(a['particles_rec'], b['particles_rec']):.3f}; "
          f"cell counts moved {moved:.2e}; total variation per sample max {tv.max():.2e}")
    # same emission up to rounding: an emission time within rounding of a
    # sample time can fall on either side of it in the two precisions
    dtot = np.abs(ga.reshape(ns, -1).sum(axis=1) - gb.reshape(ns, -1).sum(axis=1))
    print(f"  sample totals differ by at most {dtot.max()} of {n}")
    assert dtot.max() <= 10 + 1e-5 * n
    # as if independent (they are positively correlated, so this is loose)
    pv = homogeneity_pvalues(gb, ga, n, n)
    assert pv.min() > 1e-3 / ns


def test_batched_instances_fp32_error(P):
    # 16 of the batched films (particle counts capped at 2e5), the batch
    # launched in FP64 and in FP32: per instance kappa agrees within 3 sigma
    probs = [W.with_run(p, n_particles=min(p["run"]["n_particles"], 200_000)) for p in W.batched_films(256)[::16]]
    res = {}
    for prec in ("fp64", "fp32"):
        with P.Batch([W.with_run(p, precision=prec) for p in probs]) as bt:
            bt.launch()
            res[prec] = bt.results()
    rel, zs = [], []
    for ra, rb in zip(res["fp64"], res["fp32"]):
        rel.append(rb["kappa"] / ra["kappa"] - 1.0)
        zs.append(abs(rb["kappa"] - ra["kappa"]) / np.hypot(ra["kappa_se"], rb["kappa_se"]))
        assert ra["particles"] == rb["particles"]
    print(f"\nbatched films: FP32 vs FP64 kappa, median |rel. error| {np.median(np.abs(rel)):.2e}, "
          f"max {np.max(np.abs(rel)):.2e}; max z {max(zs):.2f}")
    assert max(zs) < 3.0
