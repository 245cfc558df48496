"""GPU parity on the schedule paths of the trace kernel.

The persistent kernel does not serve particles in id order when some are
emitted in modes whose mean free path far exceeds the film thickness (their
histories run to thousands of wall segments, steps III-IVa of the trajectory
algorithm repeated between relaxations):

* long-first list: particles with Lambda above long_mfp_cut (32 L) are
  listed by a classification pass and claimed, 32 at a time, before the rest;
* extreme list: those above 32 x that cut are each traced by a warp of its
  own whose idle lanes precompute its random words ("assisted rounds", a
  second inlined copy of the segment code);
* extreme-list overflow: with more extreme particles than the list holds
  (512), none is traced apart and the whole list joins the long-first list.

A gray film (one mode, so the oracle draws the same modes) with Lambda / L
chosen inside each band puts every particle on the path under test.  FP64
runs must reproduce the oracle particle by particle: sign, fate and event
counts bit-equal, the algebraic path length to 1e-12 of a mean free path
(the device fuses multiply-adds, the oracle rounds each operation).
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


def _film(n, lam, precision="fp64", schedule="auto"):
    # thickness 1, v = 1, tau = Lambda: Lambda / L = lam; K_s 12, K_e 4096
    p = W.silicon_film(n_particles=n, thickness=1.0, material=dict(W.GRAY_UNIT, tau=float(lam), v=1.0),
                       precision=precision, max_scatter=12, max_events=4096, dTdz=-1.0)
    p["run"]["schedule"] = schedule
    return p


CASES = {
    # name: (particles, Lambda / L, schedule, long-first listed, traced apart)
    "long-first list": (5000, 100.0, "auto", 5000, 0),
    "extreme list, assisted rounds": (300, 3000.0, "long_first", 0, 300),
    "extreme list overflow": (700, 3000.0, "long_first", 700, 0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_schedule_path_per_particle_fp64(P, oracle, case):
    n, lam, schedule, listed, apart = CASES[case]
    prob = _film(n, lam, schedule=schedule)
    g = P.simulate(prob, record_particles=True)
    o = oracle.run(prob, record_particles=True)
    # the path under test was the one taken
    assert g["kernel_launches"] == 2 and g["long_listed"] == listed and g["extreme_traced"] == apart
    gr, orr = g["particles_rec"], o["particles_rec"]
    for f in ("sign", "fate", "n_seg", "n_scat", "n_wall", "mode0"):
        assert np.array_equal(gr[f], orr[f]), f
    np.testing.assert_allclose(gr["L_axis"], orr["L_axis"], rtol=0, atol=1e-12 * lam)
    np.testing.assert_allclose(gr["x0"], orr["x0"], rtol=0, atol=1e-15)
    for k in ("particles", "segments", "scatters", "wall_hits", "truncated"):
        assert g[k] == o[k], k
    # long histories: most reach the segment cap
    assert np.mean(gr["n_seg"]) > 200
    assert g["kappa"] == pytest.approx(o["kappa"], rel=1e-9)
    assert g["device_flags"] == 0


def test_assisted_rounds_fp32_match_the_main_loop(P, oracle):
    # FP32: the same extreme particles traced apart (assisted rounds, the
    # long-first schedule) and in id order by the main loop follow the same
    # histories up to the compilers' contraction choices in the two inlined
    # copies, and both agree with the FP64 oracle within 3 sigma
    n, lam = 400, 3000.0
    a = P.simulate(_film(n, lam, "fp32", schedule="long_first"), record_particles=True)
    b = P.simulate(_film(n, lam, "fp32", schedule="natural"), record_particles=True)
    assert a["extreme_traced"] == n and b["kernel_launches"] == 1 and b["long_listed"] == 0
    ra, rb = a["particles_rec"], b["particles_rec"]
    same = (ra["n_seg"] == rb["n_seg"]) & (ra["fate"] == rb["fate"]) & (ra["n_scat"] == rb["n_scat"])
    print(f"\nassisted vs main loop, FP32: {np.mean(same):.4f} of histories identical")
    assert np.mean(same) > 0.9
    assert np.array_equal(ra["sign"], rb["sign"]) and np.array_equal(ra["mode0"], rb["mode0"])
    o = oracle.run(_film(20 * n, lam, "fp64"))
    for g in (a, b):
        z = abs(g["kappa"] - o["kappa"]) / np.hypot(g["kappa_se"], o["kappa_se"])
        assert z < 3.0, z


def test_schedule_does_not_change_fp64_results(P):
    # the same multi-mode film, thin enough for all three bands to occur, in
    # id order and long-first: the same particles (the assisted rounds are a
    # second inlined copy of the segment code, so path lengths may differ in
    # the last bits where the compiler fused multiply-adds differently)
    prob = W.silicon_film(n_particles=20_000, thickness=10e-9, precision="fp64")
    outs = [P.simulate(W.with_run(prob, schedule=s), record_particles=True) for s in ("natural", "long_first")]
    assert outs[0]["long_listed"] == 0 and outs[1]["long_listed"] > 0 and outs[1]["extreme_traced"] > 0
    ra, rb = outs[0]["particles_rec"], outs[1]["particles_rec"]
    for f in ("sign", "fate", "n_seg", "n_scat", "n_wall", "mode0"):
        assert np.array_equal(ra[f], rb[f]), f
    np.testing.assert_allclose(ra["L_axis"], rb["L_axis"], rtol=1e-12, atol=1e-21)
