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
