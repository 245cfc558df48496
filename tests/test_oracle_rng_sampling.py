"""Oracle pins: random stream, samplers and material tables (CPU only).

Each check compares the oracle with something other than itself: NVIDIA's
curand Philox header compiled for the host, exact probabilities, textbook
moments of the angular laws, and physical limits of the mode tables.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import stats

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def curand_host(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "curand_philox4x32_x.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("curand") / "philox_host")
    subprocess.run([cxx, "-O1", "-I", CUDA_INC, "-o", exe, os.path.join(HERE, "curand_philox_host.cpp")],
                   check=True)
    return exe


def test_philox_matches_curand_header(oracle, curand_host):
    rng = np.random.default_rng(7)
    rows = [(0, 0, 0, 0, 0, 0), (0xFFFFFFFF,) * 6, (1, 2, 3, 4, 5, 6)]
    rows += [tuple(int(x) for x in r) for r in rng.integers(0, 2 ** 32, size=(500, 6), dtype=np.uint64)]
    # the counter layout used by the tracer: (event, block, particle, instance)
    rows += [(k, b, pid, 3, 0x12063316, 0x5EED) for k in (0, 1, 4095) for b in (0, 1, 65) for pid in (0, 1, 99991)]
    inp = "\n".join(" ".join(str(v) for v in r) for r in rows) + "\n"
    out = subprocess.run([curand_host], input=inp, capture_output=True, text=True, check=True).stdout
    ref = [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]
    got = [oracle.philox(r[:4], r[4:]) for r in rows]
    assert got == ref


def test_emission_positions_uniform(oracle):
    # GRADIENT source in a film: x0 = u0 * L, so x0/L must be U(0,1)
    p = W.silicon_film(n_particles=200_000, thickness=1.0, precision="fp64")
    st, _ = oracle.emit(p, 0, 200_000)
    x = st[:, 1]
    assert np.all((x > 0) & (x < 1))
    assert stats.kstest(x, "uniform").pvalue > 1e-4
    counts, _ = np.histogram(x, bins=100, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-4


def test_wall_emission_cosine_law(oracle):
    # Isothermal wall source: V_g cos(theta) C |dT| H[cos theta] -> pdf 2 mu on ]0,1]
    p = W.gray_slab(n_particles=200_000)
    st, _ = oracle.emit(p, 0, 200_000)
    sign, x, ox, oy, oz = st[:, 0], st[:, 1], st[:, 4], st[:, 5], st[:, 6]
    lo = x == 0.0
    hi = x == 1.0
    assert np.all(lo | hi)
    assert np.all(sign[lo] == 1) and np.all(sign[hi] == -1)
    mu = np.where(lo, ox, -ox)
    assert np.all(mu > 0)
    n = mu.size
    assert abs(mu.mean() - 2 / 3) < 5 * np.sqrt(1 / 18 / n)        # E[mu] = 2/3, Var = 1/18
    assert abs((mu ** 2).mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)   # E[mu^2] = 1/2, Var = 1/12
    # CDF of mu under 2 mu dmu is mu^2, so mu^2 is uniform
    assert stats.kstest(mu ** 2, "uniform").pvalue > 1e-4
    phi = np.arctan2(oz, oy)
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4
    assert np.allclose(ox ** 2 + oy ** 2 + oz ** 2, 1.0, atol=1e-12)
    # hot and cold walls equally likely when |dT| is equal
    assert abs(lo.mean() - 0.5) < 5 * 0.5 / np.sqrt(n)


def test_gradient_emission_law_and_sign_balance(oracle):
    # Eq. 6: emission proportional to -V_g cos(theta) dT/dz: |mu_z| has pdf 2|mu|,
    # sign = sgn(-mu_z dT/dz), and equal numbers of each sign.
    p = W.silicon_film(n_particles=100_000, thickness=1e-7, precision="fp64", dTdz=-1e6)
    st, _ = oracle.emit(p, 0, 100_000)
    sign, oz = st[:, 0], st[:, 6]
    assert (sign == 1).sum() == (sign == -1).sum() == 50_000
    assert np.all(np.sign(oz) == sign)  # dT/dz < 0: s = sgn(mu_z)
    assert stats.kstest(oz ** 2, "uniform").pvalue > 1e-4
    p2 = W.silicon_film(n_particles=1000, thickness=1e-7, precision="fp64", dTdz=+1e6)
    st2, _ = oracle.emit(p2, 0, 1000)
    assert np.all(np.sign(st2[:, 6]) == -st2[:, 0])


def _merge_small(expected, observed, min_expected=20.0):
    e_out, o_out, e_acc, o_acc = [], [], 0.0, 0
    for e, o in zip(expected, observed):
        e_acc += e
        o_acc += o
        if e_acc >= min_expected:
            e_out.append(e_acc)
            o_out.append(o_acc)
            e_acc, o_acc = 0.0, 0
    if e_acc > 0:
        e_out[-1] += e_acc
        o_out[-1] += o_acc
    return np.array(e_out), np.array(o_out)


@pytest.mark.parametrize("which", ["emit", "scatter"])
def test_inverse_cdf_mode_draws(oracle, analytic, which):
    p = W.silicon_film(n_particles=1, precision="fp64")
    _, v, tau, C = analytic.mode_table(p["material"])
    w = C * v if which == "emit" else C / tau  # Eq. 2 for scattering, C v for emission
    prob = w / w.sum()
    n = 1_000_000
    u = (np.random.default_rng(11).integers(0, 2 ** 32, n, dtype=np.uint64) + 0.5) / 2.0 ** 32
    modes = oracle.draw_modes(p, which, u)
    counts = np.bincount(modes, minlength=prob.size)
    e, o = _merge_small(prob * n, counts)
    chi2 = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, len(e) - 1) > 1e-4
    # the inverse CDF is monotone in u
    order = np.argsort(u)
    assert np.all(np.diff(modes[order]) >= 0)


def test_mode_tables_match_independent_build(oracle, analytic):
    mat = W.SILICON_LIKE
    om, v, tau, C = oracle.material({"material": mat, "geometry": {"kind": "bulk"},
                                     "source": {"kind": "gradient", "dTdz": -1.0},
                                     "run": W.silicon_film(1)["run"]})
    om2, v2, tau2, C2 = analytic.mode_table(mat)
    for a, b in ((om, om2), (v, v2), (tau, tau2), (C, C2)):
        np.testing.assert_allclose(a, b, rtol=1e-12)


def test_mode_tables_physical_limits(oracle, analytic):
    mat = dict(W.SILICON_LIKE)
    om, v, tau, C = analytic.mode_table(mat)
    nb = mat["n_bins"]
    c1_la, c2_la = mat["branches"][0]["c1"], mat["branches"][0]["c2"]
    c1_ta, c2_ta = mat["branches"][1]["c1"], mat["branches"][1]["c2"]
    # group velocity -> c1 at low frequency, stays positive at the clamped TA edge
    assert abs(v[0] / c1_la - 1) < 1e-3 and abs(v[nb] / c1_ta - 1) < 1e-3
    assert np.all(v > 0)
    # TA branch is clamped at the van Hove point k = c1/(2|c2|) (just below 2 pi / a)
    assert om[2 * nb - 1] < c1_ta ** 2 / (4 * abs(c2_ta))
    assert 100.0 < v[2 * nb - 1] < 130.0
    # classical limit: sum C_b -> k_B * (modes per volume) = k_B g k_max^3 / (6 pi^2).
    # LA alone has no singular density of states, so the midpoint bins are exact to O(dw^2).
    hot_la = dict(mat, T_eq=1e7, B=0.0, branches=[mat["branches"][0]])
    k_la = 2 * np.pi / mat["a_lattice"]
    _, _, _, Ch = analytic.mode_table(hot_la)
    assert abs(Ch.sum() / (analytic.KB * k_la ** 3 / (6 * np.pi ** 2)) - 1) < 1e-5
    prob = {"material": hot_la, "geometry": {"kind": "bulk"}, "source": {"kind": "gradient", "dTdz": -1.0},
            "run": W.silicon_film(1)["run"]}
    _, _, _, Co = oracle.material(prob)
    assert abs(Co.sum() / (analytic.KB * k_la ** 3 / (6 * np.pi ** 2)) - 1) < 1e-5
    # TA is clamped at its van Hove point, where D ~ (w_max - w)^-1/2: the midpoint bins
    # under-count the last bin, an error that must shrink like n_bins^-1/2.
    k_ta = c1_ta / (2 * abs(c2_ta))
    ref_ta = 2 * k_ta ** 3 / (6 * np.pi ** 2)
    errs = []
    for nbins in (1000, 16000):
        hot_ta = dict(mat, T_eq=1e7, B=0.0, branches=[mat["branches"][1]], n_bins=nbins)
        _, _, _, Ct = analytic.mode_table(hot_ta)
        errs.append(1 - Ct.sum() / (analytic.KB * ref_ta))
    assert 0 < errs[0] < 0.1 and 0 < errs[1] < errs[0] / 3.5
    # Rayleigh-type scattering rate at fixed frequency scales as omega^4 when B = 0
    _, _, t1, _ = analytic.mode_table(dict(mat, B=0.0))
    assert abs((t1[0] / t1[1]) / ((om[1] / om[0]) ** 4) - 1) < 1e-12
