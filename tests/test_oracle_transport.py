"""Oracle pins: full trajectories against closed forms and exact invariants.

* gray slab between black walls: heat flux and bin-averaged temperature
  against the deterministic integral-equation solution (``analytic``);
  ballistic limit; per-particle telescoping s L_x / L in {0, 1}; the per-bin
  flux equals the total flux exactly; every particle is absorbed.
* films with diffuse walls: conductivity against the Fuchs-Sondheimer sum,
  bulk conductivity against (1/3) sum C v^2 tau, and the vanishing mean
  contribution after the first event (first-event truncation is exact for
  the film, scattering-index tallies H_j, j >= 1, average to zero).
"""
import math
import numpy as np
import pytest

import workloads as W


def _z(a, b, se):
    return abs(a - b) / se


@pytest.mark.parametrize("kn,n", [(1.0, 400_000), (0.5, 200_000), (2.0, 200_000)])
def test_gray_slab_psi_against_integral_equation(oracle, analytic, kn, n):
    r = oracle.run(W.gray_slab(n_particles=n, kn=kn, n_bins=0))
    pin = analytic.slab_solution(1.0 / kn, n_bins=50, M=200)["psi"]
    # Psi is a Bernoulli mean (each particle crosses or not): sigma^2 = Psi(1-Psi)/N
    se = np.sqrt(pin * (1 - pin) / n)
    assert _z(r["psi"], pin, se) < 4.0
    assert r["absorbed"] == n and r["truncated"] == 0


def test_gray_slab_temperature_profile(oracle, analytic):
    n = 400_000
    r = oracle.run(W.gray_slab(n_particles=n, kn=1.0, n_bins=50))
    ref = analytic.slab_solution(1.0, n_bins=50, M=200)
    z = (r["T"] - ref["T_bins"]) / r["T_se"]
    assert np.max(np.abs(z)) < 5.0
    assert np.mean(z ** 2) < 2.0
    # antisymmetry of T(x) - T_eq about the mid-plane, within noise
    anti = (r["T"] + r["T"][::-1]) / np.sqrt(r["T_se"] ** 2 + r["T_se"][::-1] ** 2)
    assert np.max(np.abs(anti)) < 5.0
    # every bin carries exactly the total flux (per-particle telescoping in each bin)
    assert np.allclose(r["q"], r["flux"], rtol=1e-9, atol=0)


def test_gray_slab_ballistic_limit(oracle):
    n = 50_000
    r = oracle.run(W.gray_slab(n_particles=n, tau=1e30, n_bins=10), record_particles=True)
    assert r["psi"] == pytest.approx(1.0, abs=1e-12)
    rec = r["particles_rec"]
    assert np.all(rec["n_scat"] == 0) and np.all(rec["n_seg"] == 1)


def test_gray_slab_per_particle_invariants(oracle):
    n = 20_000
    r = oracle.run(W.gray_slab(n_particles=n, kn=1.0, n_bins=0), record_particles=True)
    rec = r["particles_rec"]
    sl = rec["sign"] * rec["L_axis"]
    frac = np.minimum(np.abs(sl - 0.0), np.abs(sl - 1.0))
    assert np.max(frac) < 1e-12                      # s L_x / L in {0, 1}
    assert np.all(rec["fate"] == 0)                  # absorbed
    assert np.all(rec["n_seg"] == rec["n_scat"] + 1)  # one wall event ends each life
    assert np.all(rec["n_wall"] == 1)
    assert r["psi"] == pytest.approx(np.mean(np.round(sl)), abs=1e-12)


def test_gray_film_first_event_is_exact(oracle, analytic):
    # Lambda = L: kappa / kappa_bulk = S(1).  Truncating after the first event
    # (wall or scattering) is exact for the diffuse film; so is the full run.
    mat = dict(W.GRAY_UNIT)
    kb = 1.0 / 3.0
    s1 = float(analytic.fuchs_sondheimer(1.0))
    for max_events, n in ((1, 2_000_000), (4096, 400_000)):
        p = W.silicon_film(n_particles=n, thickness=1.0, material=mat, precision="fp64",
                           max_scatter=40, max_events=max_events, dTdz=-1.0)
        r = oracle.run(p)
        assert _z(r["kappa"], kb * s1, r["kappa_se"]) < 4.0, (max_events, r["kappa"], kb * s1)


def test_silicon_film_fuchs_sondheimer(oracle, analytic):
    mat = W.SILICON_LIKE
    for L, n in ((100e-9, 4_000_000), (1e-6, 2_000_000)):
        pin = analytic.kappa_film(mat, L)
        r = oracle.run(W.silicon_film(n_particles=n, thickness=L, precision="fp64", max_events=1))
        assert _z(r["kappa"], pin, r["kappa_se"]) < 4.0, (L, r["kappa"], pin)
    # full trajectories with the 40-scattering cap: still unbiased for the film
    pin = analytic.kappa_film(mat, 100e-9)
    r = oracle.run(W.silicon_film(n_particles=1_000_000, thickness=100e-9, precision="fp64"))
    assert _z(r["kappa"], pin, r["kappa_se"]) < 4.0, (r["kappa"], pin)


def test_specular_film_factor_forms(analytic):
    # the first-flight derivation and the usual t-integral agree, reduce to the
    # diffuse closed form at p = 0 and to the bulk (S = 1) at p = 1
    for d in (0.02, 0.3, 1.0, 4.0):
        assert analytic.fuchs_sondheimer_specular(d, 0.0) == pytest.approx(float(analytic.fuchs_sondheimer(d)),
                                                                           rel=1e-10)
        assert analytic.fuchs_sondheimer_specular(d, 1.0) == pytest.approx(1.0, rel=1e-12)
        for p in (0.25, 0.6):
            assert analytic.fuchs_sondheimer_specular(d, p) == pytest.approx(
                analytic.fuchs_sondheimer_specular_t(d, p), rel=1e-9)


def test_partially_specular_film(oracle, analytic):
    # Walls specular with probability p (the rest diffuse): Fuchs-Sondheimer
    # with specularity p.  Truncation stays unbiased: a relaxation or a diffuse
    # hit leaves a zero mean in-plane velocity, and 4096 segments without a
    # diffuse hit have probability p^4096.
    mat = W.SILICON_LIKE
    pin = analytic.kappa_film(mat, 100e-9, 0.25)
    r = oracle.run(W.silicon_film(n_particles=4_000_000, precision="fp64", specularity=0.25))
    assert _z(r["kappa"], pin, r["kappa_se"]) < 4.0, (r["kappa"], pin)
    # the pin tells this specularity from its complement and from diffuse walls
    assert abs(analytic.kappa_film(mat, 100e-9, 0.75) - pin) > 10 * r["kappa_se"]
    assert abs(analytic.kappa_film(mat, 100e-9) - pin) > 10 * r["kappa_se"]
    # fully specular walls never end an in-plane flight: the bulk value
    gray = dict(W.GRAY_UNIT)
    r = oracle.run(W.silicon_film(n_particles=1_000_000, thickness=1.0, material=gray, precision="fp64",
                                  specularity=1.0, dTdz=-1.0, max_scatter=1, max_events=1 << 20))
    assert _z(r["kappa"], 1.0 / 3.0, r["kappa_se"]) < 4.0


def test_first_collision_truncation(oracle, analytic):
    # Stopping at the first relaxation or wall hit (the first free path) is
    # exact for the diffuse film; every particle then has exactly one segment.
    pin = analytic.kappa_film(W.SILICON_LIKE, 100e-9)
    r = oracle.run(W.with_run(W.silicon_film(n_particles=2_000_000, precision="fp64"), max_collisions=1))
    assert _z(r["kappa"], pin, r["kappa_se"]) < 4.0, (r["kappa"], pin)
    assert r["segments"] == r["particles"] == r["truncated"]
    # In the pored film a pore wall re-emits a particle back against the flux
    # on average, so following only the first free path (crossings of the
    # periodic unit-cell faces do not end it) overestimates the conductivity.
    full = oracle.run(W.porous_film(n_particles=400_000, precision="fp64"))
    first = oracle.run(W.with_run(W.porous_film(n_particles=400_000, precision="fp64"), max_collisions=1))
    assert first["periodic"] > 0 and first["scatters"] + first["wall_hits"] == first["particles"]
    assert first["kappa"] - full["kappa"] > 5.0 * math.hypot(first["kappa_se"], full["kappa_se"])


@pytest.mark.parametrize("g", [0.6, -0.4])
def test_anisotropic_scattering_direction_law(oracle, g):
    # Henyey-Greenstein about the incoming direction: unit vectors, cosine
    # distributed by the law's CDF (mean g), azimuth about the incoming
    # direction uniform in a frame built here independently
    from scipy import stats
    rng = np.random.default_rng(7)
    n = 4000
    inc = rng.normal(size=(n, 3))
    inc /= np.linalg.norm(inc, axis=1)[:, None]
    inc[0] = (0.0, 0.0, 1.0)
    inc[1] = (0.0, 0.0, -1.0)
    u = (rng.integers(0, 2 ** 32, size=(n, 2)).astype(np.float64) + 0.5) / 2.0 ** 32
    out = np.array([oracle.scatter_direction(g, inc[i], u[i, 0], u[i, 1]) for i in range(n)])
    assert np.allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-12)
    mu = np.sum(out * inc, axis=1)
    cdf = lambda m: (1 - g * g) / (2 * g) * ((1 + g * g - 2 * g * np.clip(m, -1, 1)) ** -0.5 - 1 / (1 + g))
    assert stats.kstest(mu, cdf).pvalue > 1e-3
    e = np.where(np.abs(inc[:, :1]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    t1 = np.cross(inc, e)
    t1 /= np.linalg.norm(t1, axis=1)[:, None]
    t2 = np.cross(inc, t1)
    phi = np.arctan2(np.sum(out * t2, axis=1), np.sum(out * t1, axis=1))
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-3


def test_isotropic_law_is_g_zero(oracle):
    # g = 0 keeps the paper's isotropic redraw: mu_z = 2u - 1, whatever the incoming direction
    out = oracle.scatter_direction(0.0, [1.0, 0.0, 0.0], 0.8, 0.25)
    assert out[2] == pytest.approx(0.6, abs=1e-15)


def test_anisotropic_bulk_conductivity(oracle, analytic):
    mat = dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0, scatter_g=0.5)
    r = oracle.run(W.bulk(n_particles=400_000, material=mat))
    assert _z(r["kappa"], 7.0 * 9.0 * 2.5 / 3.0 / 0.5, r["kappa_se"]) < 4.0
    assert analytic.kappa_bulk_anisotropic(mat, 0.5) == pytest.approx(7.0 * 9.0 * 2.5 / 3.0 / 0.5, rel=1e-14)
    si = dict(W.SILICON_LIKE, scatter_g=0.4)
    pin = analytic.kappa_bulk_anisotropic(si, 0.4)
    r = oracle.run(W.bulk(n_particles=2_000_000, material=si))
    assert _z(r["kappa"], pin, r["kappa_se"]) < 4.0, (r["kappa"], pin)
    assert abs(pin - analytic.kappa_bulk(W.SILICON_LIKE)) > 10 * r["kappa_se"]


def test_anisotropic_flux_split_is_geometric(oracle):
    # gray bulk: the mean flux between relaxation j and j + 1 is g^j times the first flight's
    g = 0.6
    mat = dict(W.GRAY_UNIT, scatter_g=g)
    p = W.bulk(n_particles=1_000_000, material=mat, dTdz=-1.0)
    p["run"]["n_hj"] = 8
    r = oracle.run(p)
    H, se = r["H"], r["H_se"]
    for j in range(1, 7):
        ratio = H[j] / H[0]
        err = abs(ratio) * np.hypot(se[j] / H[j], se[0] / H[0])
        assert abs(ratio - g ** j) < 4.0 * err + 1e-12, (j, ratio, g ** j, err)


def test_bulk_first_flight_second_moment(oracle):
    # First flight only (max_events = 1) in a gray bulk: s L_z = l mu with
    # l ~ Exp(Lambda) and mu from the |mu| law, so E[(s L_z)^2] = 2 Lambda^2 / 2
    # = Lambda^2 and Var((s L_z)^2) = E[l^4] E[mu^4] - Lambda^4 = 7 Lambda^4.
    # The conductivity pins only see the mean flight; this one sees its shape.
    lam, n = 2.5 * 3.0, 1_000_000
    r = oracle.run(W.bulk(n_particles=n, material=dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0), max_events=1))
    m2 = r["sum_sL2"] / n
    assert abs(m2 - lam ** 2) < 4.0 * math.sqrt(7.0 / n) * lam ** 2, (m2, lam ** 2)


def test_bulk_conductivity(oracle, analytic):
    # no boundaries: kappa = (1/3) sum C v^2 tau exactly in expectation
    mat = dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0)
    r = oracle.run(W.bulk(n_particles=2_000_000, material=mat, max_events=8))
    assert _z(r["kappa"], 7.0 * 9.0 * 2.5 / 3.0, r["kappa_se"]) < 4.0
    r = oracle.run(W.bulk(n_particles=4_000_000, max_events=1))
    assert _z(r["kappa"], analytic.kappa_bulk(W.SILICON_LIKE), r["kappa_se"]) < 4.0


def test_contributions_after_first_scattering_vanish(oracle):
    # Diffuse film, isotropic scattering: <H_j> = 0 for j >= 1 (expected value of
    # V_g . e_z after a scattering is zero), and sum_j H_j equals the flux.
    p = W.silicon_film(n_particles=400_000, thickness=100e-9, precision="fp64", n_hj=41)
    r = oracle.run(p)
    H, Hse = r["H"], r["H_se"]
    assert np.isclose(H.sum(), r["flux"], rtol=1e-9)
    z = H[1:] / np.where(Hse[1:] > 0, Hse[1:], 1.0)
    assert np.max(np.abs(z)) < 5.0
    assert H[0] > 10 * Hse[0]


def test_truncation_counts(oracle):
    p = W.silicon_film(n_particles=20_000, thickness=100e-9, precision="fp64", max_scatter=5, max_events=64)
    r = oracle.run(p, record_particles=True)
    rec = r["particles_rec"]
    assert np.all((rec["fate"] == 1) | (rec["fate"] == 2))
    assert np.all(rec["n_seg"] <= 64) and np.all(rec["n_scat"] <= 5)
    assert np.all(rec["n_seg"] == rec["n_scat"] + rec["n_wall"])
    assert np.all((rec["fate"] != 1) | (rec["n_scat"] == 5))
    assert np.all((rec["fate"] != 2) | (rec["n_seg"] == 64))
    assert r["truncated"] == 20_000


def test_nongray_slab_against_collision_density_solution(oracle, analytic):
    # Pins the emission law (C v, cosine) and Eq. 2 (C / tau) together with the
    # per-mode mean free paths: a black-walled silicon-like slab, 20 modes.
    mat = dict(W.SILICON_LIKE, n_bins=10)
    L = 100e-9
    _, v, tau, C = analytic.mode_table(mat)
    lam = v * tau
    pin = analytic.slab_multimode_psi(lam, C * v, C / tau, L, M=100)
    p = W.gray_slab(n_particles=1_000_000, n_bins=0)
    p["material"] = mat
    p["geometry"]["L"] = L
    r = oracle.run(p)
    assert abs(r["psi"] - pin) < 4.0 * r["psi_se"], (r["psi"], pin)
    # the pin discriminates: redrawing modes from C v instead of Eq. 2 moves Psi by >> 4 sigma
    wrong = analytic.slab_multimode_psi(lam, C * v, C * v, L, M=100)
    assert abs(wrong - pin) > 20.0 * r["psi_se"]


def test_two_slab_solvers_agree(analytic):
    # emissive-power and collision-density formulations of the gray slab
    for tau_L in (0.5, 1.0, 2.0):
        a = analytic.slab_solution(tau_L, M=200)["psi"]
        b = analytic.slab_multimode_psi([1.0 / tau_L], [1.0], [1.0], 1.0, M=100)
        assert abs(a - b) < 5e-6
    # the exact flux is the same at every interior plane
    q = analytic.slab_flux_profile(1.0, [0.1, 0.3, 0.5, 0.7, 0.9], M=200)
    assert np.ptp(q) < 1e-5
    # thin limit: Psi -> 1/2 + E3(tau_L) to first order (phi ~ 1/2 inside)
    t = 0.02
    assert abs(analytic.slab_solution(t, M=200)["psi"] - (0.5 + float(analytic.En(3, t)))) < 1e-3
    # thick limit approaches the diffusion result with jump conditions, 4/(3 tau_L + 4)
    assert abs(analytic.slab_solution(50.0, M=400)["psi"] / (4.0 / (3 * 50.0 + 4.0)) - 1) < 0.01


def test_truncation_study_predicts_dropped_flux(oracle, built_library):
    # Pored film, flux split by scattering index up to 64 relaxations: the
    # geometric extrapolation of the resolved, decaying <H_j> predicts the flux
    # a cap K drops (measured directly as the sum of the later <H_j>) within
    # the statistical error of that sum; the paper's noise criterion gives K_s.
    # (The study is the library's host-only arithmetic, fed the oracle's split.)
    study = built_library.truncation_study
    p = W.porous_film(n_particles=2_000_000, precision="fp64", max_scatter=64, n_hj=64)
    r = oracle.run(p)
    H, se = r["H"], r["H_se"]
    st = study(H, se)
    assert 3 <= st["k_s"] < 64 and 0.0 < st["ratio"] < 1.0
    for K in (2, 4, 6):
        dropped, err = H[K:].sum(), np.sqrt((se[K:] ** 2).sum())
        assert abs(st["tail"](K) - dropped) < 3.0 * err, (K, st["tail"](K), dropped, err)
    # diffuse film: nothing after the first event survives in expectation
    f = oracle.run(W.silicon_film(n_particles=400_000, precision="fp64", n_hj=16))
    sf = study(f["H"], f["H_se"])
    assert sf["k_s"] <= 3 and np.all(np.abs(f["H"][1:]) < 4.0 * f["H_se"][1:])


def film_profile_pvalues(oracle, analytic, L=40e-9, lam=2e-8, n=400_000, library=None):
    """chi-square p-values of a gray film's depth profiles under the gradient
    source: the in-plane flux q_z(x) against the depth form of the
    Fuchs-Sondheimer solution, and T(x) against zero (no deviational
    temperature in a uniformly driven film)."""
    from scipy import stats
    mat = dict(W.GRAY_UNIT, tau=lam, v=1.0)
    p = W.silicon_film(n_particles=n, thickness=L, material=mat, precision="fp64", dTdz=-1e6, max_scatter=40)
    p["run"].update(n_bins_x=10, n_batch=16)
    o = oracle.run(p, library=library)
    pin = analytic.film_flux_profile(mat, L, 10, dTdz=-1e6)
    zq = (o["q"] - pin) / o["q_se"]
    zT = o["T"] / o["T_se"]
    assert np.mean(o["q"]) == pytest.approx(o["flux"], rel=1e-12)  # the bins partition the flux
    return stats.chi2.sf(np.sum(zq ** 2), zq.size), stats.chi2.sf(np.sum(zT ** 2), zT.size)


@pytest.mark.parametrize("L", [40e-9, 10e-9])
def test_film_in_plane_flux_by_depth(oracle, analytic, L):
    # the depth form of the thin-film solution: its slab means average to the
    # Fuchs-Sondheimer factor, and the oracle's q_z(x) follows it bin by bin
    assert np.mean(analytic.film_flux_profile(W.SILICON_LIKE, 100e-9, 20)) / 1e6 == pytest.approx(
        analytic.kappa_film(W.SILICON_LIKE, 100e-9), rel=1e-6)
    pq, pT = film_profile_pvalues(oracle, analytic, L=L)
    assert pq > 1e-3 and pT > 1e-3, (pq, pT)
