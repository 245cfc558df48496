"""GPU parity for the steady maps of the pored film: T - T_eq(z) and the z
flux over the solid of each cell of a (y, z) map of the unit cell.

* FP64 single-mode runs give the oracle's maps cell by cell, to rounding
  (same particles, same cell crossings);
* FP32 silicon-like maps agree with the oracle's within their errors
  (chi-square), partition the scalar flux, and keep the unit cell's mirror
  symmetries;
* descriptors the maps do not apply to are rejected.
"""
import numpy as np
import pytest

import workloads as W
from tests.test_oracle_porous import map_symmetry_pvalues

pytestmark = pytest.mark.gpu

GRAY_FAST = dict(W.GRAY_UNIT, tau=2e-8, v=1.0)


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def test_gray_maps_per_particle(P, oracle):
    prob = W.porous_film(n_particles=20_000, precision="fp64", material=GRAY_FAST, max_events=300,
                         max_scatter=20, map=(8, 8), n_batch=16)
    g = P.simulate(prob)
    o = oracle.run(prob)
    assert g["segments"] == o["segments"] and g["periodic"] == o["periodic"]
    np.testing.assert_allclose(g["map_solid"], o["map_solid"], rtol=0, atol=1e-12)
    for k in ("map_T", "map_T_se", "map_q", "map_q_se"):
        a, b = g[k], o[k]
        assert np.array_equal(np.isnan(a), np.isnan(b)), k
        m = np.isfinite(b)
        # summation order, and path lengths that differ by rounding at
        # near-tangent pore hits (1e-6 of a mean free path at most)
        np.testing.assert_allclose(a[m], b[m], rtol=1e-9, atol=1e-6 * np.abs(b[m]).max(), err_msg=k)


def test_silicon_maps_against_oracle(P, oracle):
    from scipy import stats
    g = P.simulate(W.porous_film(n_particles=20_000_000, map=(8, 8), n_batch=32))
    o = oracle.run(W.porous_film(n_particles=400_000, precision="fp64", map=(8, 8), n_batch=16))
    for k in ("map_T", "map_q"):
        z = (g[k] - o[k]) / np.hypot(g[k + "_se"], o[k + "_se"])
        z = z[np.isfinite(z)]
        assert stats.chi2.sf(np.sum(z ** 2), z.size) > 1e-3, (k, np.round(z, 2))
    # the z displacements over the cells add up to the scalar flux (FP32
    # segment products summed in two different orders)
    V = g["map_solid"] * (100e-9 / 8) ** 2 * 300e-9
    assert np.nansum(g["map_q"] * V) == pytest.approx(g["flux"] * (100e-9) ** 2 * 300e-9, rel=1e-5)
    assert min(map_symmetry_pvalues(g)) > 1e-3, map_symmetry_pvalues(g)
    assert g["device_flags"] == 0
    # the local temperature adds the imposed T_eq(z): it falls along z, is odd
    # about the mid-plane, and the deviation bends it around the pore
    zc = (np.arange(8) + 0.5) * (100e-9 / 8) - 50e-9
    has = g["map_solid"] > 0
    assert np.array_equal(np.isnan(g["map_T_local"]), ~has)
    np.testing.assert_allclose((g["map_T_local"] - g["map_T"])[has], ((zc * -1e7)[:, None] * np.ones((1, 8)))[has],
                               rtol=1e-12, atol=1e-12)
    rows = np.nanmean(g["map_T_local"], axis=1)
    assert np.all(np.diff(rows) < 0)
    np.testing.assert_allclose(g["map_T_local"], -g["map_T_local"][::-1, :], atol=6 * np.nanmax(g["map_T_se"]))
    print(f"\nmap T range {np.nanmin(g['map_T']):.3f} .. {np.nanmax(g['map_T']):.3f} K, "
          f"q_z range {np.nanmin(g['map_q']):.3e} .. {np.nanmax(g['map_q']):.3e} W/m^2, "
          f"largest T error {np.nanmax(g['map_T_se']):.4f} K")


def test_map_descriptors_rejected(P):
    bad = [W.with_run(W.silicon_film(n_particles=1000), map=(4, 4)),   # no pores
           W.with_run(W.porous_pulse(n_particles=1000), map=(4, 4)),   # transient
           W.porous_film(n_particles=1000, map=(65, 4)),               # too many cells per axis
           W.porous_film(n_particles=1000, map=(8, 8), n_batch=65),    # too many batch groups
           W.with_run(W.porous_film(n_particles=1000), map=(4, 0))]    # one axis only
    for prob in bad:
        with pytest.raises(P.LeMcError) as e:
            P.simulate(prob)
        assert e.value.status == 1


def test_map_size_limits(P):
    # one cell: the map is the whole unit cell, so its flux is the solid-averaged
    # scalar flux; the largest map and batch count stay consistent too
    g = P.simulate(W.porous_film(n_particles=200_000, map=(1, 1), n_batch=64))
    solid = 1.0 - np.pi * 0.3 ** 2
    assert g["map_solid"][0, 0] == pytest.approx(solid, rel=1e-12)
    assert g["map_q"][0, 0] == pytest.approx(g["flux"] / solid, rel=1e-5)
    big = P.simulate(W.porous_film(n_particles=200_000, map=(64, 64), n_batch=64))
    V = big["map_solid"] * (100e-9 / 64) ** 2 * 300e-9
    assert np.nansum(big["map_q"] * V) == pytest.approx(big["flux"] * (100e-9) ** 2 * 300e-9, rel=1e-5)
    has = big["map_solid"] > 0
    assert np.all(np.isfinite(big["map_T"][has])) and np.all(np.isnan(big["map_T"][~has]))
    assert big["segments"] == g["segments"] and big["device_flags"] == 0


def test_fine_map_aggregates_to_coarse(P):
    # The same particles mapped on 16 x 16 and on 8 x 8 cells: each coarse
    # cell's sums are the sums over its 2 x 2 fine cells.  With 32 batch
    # groups the coarse maps (4096 entries) collect in the kernel's FP32
    # shared-memory copy and the fine ones (16384) go straight to the FP64
    # sums, so the two accumulation paths are checked against each other.
    fine = P.simulate(W.porous_film(n_particles=2_000_000, map=(16, 16), n_batch=32))
    coarse = P.simulate(W.porous_film(n_particles=2_000_000, map=(8, 8), n_batch=32))
    assert fine["segments"] == coarse["segments"] and fine["device_flags"] == coarse["device_flags"] == 0
    for k in ("map_T", "map_q"):
        vf = np.nan_to_num(fine[k] * fine["map_solid"]) * (1.0 / 16) ** 2
        vc = np.nan_to_num(coarse[k] * coarse["map_solid"]) * (1.0 / 8) ** 2
        agg = vf.reshape(8, 2, 8, 2).sum(axis=(1, 3))
        # (FP32 crossing parameters differ by rounding between the two grids)
        np.testing.assert_allclose(agg, vc, rtol=1e-4, atol=1e-5 * np.abs(vc).max(), err_msg=k)
