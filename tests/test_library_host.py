"""CPU tests of the CUDA library's host side: it loads without a GPU, exports
every entry point that include/le_mc.h declares, its structs match the
binding, and its host logic (mode tables, alias tables, validation) agrees
with the oracle and with exact probabilities.  No compute call needs a GPU."""
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P(built_library):
    return built_library


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^LE_MC_API\s+[\w\s\*]+?\b(le_mc_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(P):
    declared = _declared_functions()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(P.lib, name), name
    # and the binding wraps each of them
    from paper_1206_3316_gb300 import _binding
    assert set(declared) <= set(_binding.SIGNATURES)


def test_struct_layouts(P):
    from paper_1206_3316_gb300 import _binding as Bd
    import ctypes
    for i, cls in enumerate((Bd.MaterialDesc, Bd.GeometryDesc, Bd.RunDesc, Bd.Tallies, Bd.Particle)):
        assert P.lib.le_mc_struct_size(i) == ctypes.sizeof(cls)
    assert Bd.PARTICLE_DTYPE.itemsize == ctypes.sizeof(Bd.Particle)
    assert P.le_mc_abi_version() == 5


def test_no_device_is_reported_not_faked(P):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.LeMcError) as e:
        P.le_mc_create_material(P.material_desc(W.GRAY_UNIT))
    assert e.value.status in (3, 7)


def test_mode_table_matches_oracle(P, oracle):
    for mat in (W.SILICON_LIKE, dict(W.SILICON_LIKE, T_eq=120.0, n_bins=333), W.GRAY_UNIT):
        om, v, tau, C = P.le_mc_material_table(P.material_desc(mat))
        prob = {"material": mat, "geometry": {"kind": "bulk"}, "source": {"kind": "gradient", "dTdz": -1.0},
                "run": W.silicon_film(1)["run"]}
        o = oracle.material(prob)
        for a, b in zip((om, v, tau, C), o):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def _alias_pdf(thr, al):
    n = thr.size
    keep = thr.astype(np.float64) / 2.0 ** 32
    keep[thr == 0xFFFFFFFF] = 1.0
    pdf = np.zeros(n)
    np.add.at(pdf, np.arange(n), keep / n)
    np.add.at(pdf, al, (1.0 - keep) / n)
    return pdf


@pytest.mark.parametrize("which", ["emit", "scatter", "random", "one", "spiky"])
def test_alias_table_is_exact(P, analytic, which):
    rng = np.random.default_rng(5)
    if which in ("emit", "scatter"):
        _, v, tau, C = analytic.mode_table(W.SILICON_LIKE)
        w = C * v if which == "emit" else C / tau
    elif which == "random":
        w = rng.exponential(size=777)
    elif which == "one":
        w = np.array([3.0])
    else:
        w = np.zeros(64)
        w[[0, 17, 63]] = [1e-12, 1.0, 5.0]
    thr, al = P.le_mc_alias_table(w)
    assert np.all(al < w.size)
    pdf = _alias_pdf(thr, al)
    np.testing.assert_allclose(pdf, w / w.sum(), rtol=0, atol=2.0 ** -31)
    assert abs(pdf.sum() - 1.0) < 1e-12


def test_alias_draw_rule_reproduces_pdf(P):
    # the device rule on every (column, low-word) cell of a coarse grid of words
    w = np.array([0.1, 0.0, 2.5, 1.0, 0.4])
    thr, al = P.le_mc_alias_table(w)
    words = (np.arange(1 << 16, dtype=np.uint64) << np.uint64(16)) + np.uint64(0x7FFF)
    m = words * np.uint64(w.size)
    j = (m >> np.uint64(32)).astype(np.int64)
    lo = (m & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    modes = np.where(lo < thr[j].astype(np.uint64), j, al[j])
    freq = np.bincount(modes, minlength=w.size) / words.size
    np.testing.assert_allclose(freq, w / w.sum(), atol=5e-5)
    assert freq[1] == 0.0


def test_invalid_descriptors_rejected(P):
    bad_geo = [
        {"kind": "planes", "L": 0.0},
        {"kind": "planes", "L": float("nan")},
        {"kind": "porous", "L": 1.0, "pitch": 1.0, "radius": 0.6},
        {"kind": "porous", "L": 1.0, "pitch": 1.0, "radius": 0.2, "pore_wall": "black"},
        {"kind": "porous", "L": 1.0, "pitch": 1.0, "radius": 0.2, "cells_y": 0},
        {"kind": "planes", "L": 1.0, "wall_lo": "partial", "spec_lo": 1.5},
        {"kind": "planes", "L": 1.0, "spec_hi": -0.1},
        {"kind": "porous", "L": 1.0, "pitch": 1.0, "radius": 0.2, "pore_wall": "partial", "spec_pore": float("nan")},
    ]
    for g in bad_geo:
        with pytest.raises(P.LeMcError) as e:
            P.le_mc_create_geometry(P.geometry_desc(g))
        assert e.value.status == 1, g
    h = P.le_mc_create_geometry(P.geometry_desc({"kind": "planes", "L": 1e-7}))
    P.le_mc_destroy_geometry(h)
    bad_mat = [dict(W.GRAY_UNIT, tau=0.0), dict(W.SILICON_LIKE, n_bins=5000), dict(W.SILICON_LIKE, T_eq=-1.0),
               dict(W.GRAY_UNIT, scatter_g=1.0), dict(W.GRAY_UNIT, scatter_g=float("nan"))]
    for m in bad_mat:
        with pytest.raises(P.LeMcError) as e:
            P.le_mc_material_table(P.material_desc(m))
        assert e.value.status == 1
    with pytest.raises(P.LeMcError):
        P.le_mc_alias_table(np.zeros(4))
    with pytest.raises(P.LeMcError):
        P.le_mc_alias_table(np.array([1.0, -1.0]))


def test_map_solid_fractions_match_oracle(P, oracle):
    # two independent computations of each map cell's solid: the library's
    # closed form (inclusion-exclusion of disk-corner areas) and the oracle's
    # Gauss-Legendre quadrature of the pore's chords
    for ny, nz, r in ((8, 8, 30e-9), (16, 16, 30e-9), (7, 5, 45e-9), (64, 64, 10e-9), (3, 1, 0.0)):
        prob = W.porous_film(n_particles=64, precision="fp64", map=(ny, nz), radius=r)
        lib = P.le_mc_map_solid(P.geometry_desc(prob["geometry"]), ny, nz)
        np.testing.assert_allclose(lib, oracle.run(prob)["map_solid"], rtol=0, atol=1e-12)
    g = P.geometry_desc(W.porous_film(n_particles=1)["geometry"])
    for ny, nz in ((0, 4), (4, 65)):
        with pytest.raises(P.LeMcError):
            P.le_mc_map_solid(g, ny, nz)
    with pytest.raises(P.LeMcError):
        P.le_mc_map_solid(P.geometry_desc({"kind": "planes", "L": 1e-7}), 4, 4)


def test_truncation_study_exact_and_against_independent_fit(P):
    # An exactly geometric split is recovered exactly: ratio, amplitude, the
    # tail sum_{j >= K} H_j in closed form, and K_s where the terms fall to
    # their standard errors.
    j = np.arange(40)
    H = -3.0 * 0.5 ** j
    se = np.full(40, 3.0 * 0.5 ** 12)
    st = P.truncation_study(H, se, resolved=3.0, first=2)
    assert st["k_s"] == 12  # |H_12| == se
    assert st["ratio"] == pytest.approx(0.5, rel=1e-12)
    for K in (2, 5, 9):
        assert st["tail"](K) == pytest.approx(-3.0 * 0.5 ** K / (1 - 0.5), rel=1e-12)
    # noisy split: the fit equals numpy's weighted least squares on the same run
    rng = np.random.Generator(np.random.PCG64(7))
    H = 2.0 * 0.7 ** j * (1 + 0.05 * rng.standard_normal(40))
    se = 0.02 * np.ones(40)
    st = P.truncation_study(H, se, resolved=3.0, first=2)
    run = [k for k in range(2, 40)]
    stop = next(k for k in run if not abs(H[k]) > 3.0 * se[k])
    idx = np.arange(2, stop)
    w = (H[idx] / se[idx]) ** 2
    A = np.vstack([np.ones(idx.size), idx]).T * np.sqrt(w)[:, None]
    c = np.linalg.lstsq(A, np.log(np.abs(H[idx])) * np.sqrt(w), rcond=None)[0]
    assert st["n_fit"] == idx.size
    assert st["ratio"] == pytest.approx(np.exp(c[1]), rel=1e-10)
    assert st["tail"](6) == pytest.approx(np.exp(c[0]) * np.exp(c[1]) ** 6 / (1 - np.exp(c[1])), rel=1e-9)
    # nothing resolved beyond `first`: no fit, no extrapolated tail
    st = P.truncation_study([1.0, 0.5, 0.01, 0.0], [0.1, 0.1, 0.1, 0.1])
    assert st["ratio"] is None and st["tail"](2) == 0.0 and st["k_s"] == 2
    with pytest.raises(P.LeMcError):
        P.truncation_study([1.0, np.nan], [0.1, 0.1])
