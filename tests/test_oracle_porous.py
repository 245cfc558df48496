"""Oracle pins for the periodic porous film and the transient estimator.

* ray / boundary distances against brute-force marching with bisection;
* a porous film with zero pore radius is a plain film: its conductivity
  must equal the Fuchs-Sondheimer value, so the periodic unit-cell faces
  (which end segments and re-insert particles) change nothing;
* pores only lower the conductivity (kappa_eff below the pore-free film);
* Eq. 3 transient counts conserve energy exactly: every adiabatic-walled
  particle alive at a sample time sits in exactly one grid cell;
* steady maps over the unit cell: the solid fraction of each map cell
  (exact total, point counts), the flux map partitions the scalar flux
  exactly, the mirror symmetries of the unit cell (T odd in z about the
  pore, even in y; the z flux even in both), and the flat maps of a film
  without pores;
* free streaming between specular faces: an initial excess that never
  relaxes spreads as the folded kinematics predict slab by slab and sample
  by sample (the Eq. 3 positions interpolated at the sample times);
* surface pulse lateral law and directions: without pores the emitted
  positions are a 2-D Gaussian about (y0, z0), so r^2 / (2 sigma^2) is
  exponential (KS), and directions follow the cosine law into the film
  (|mu_x|^2 uniform, KS);
* surface pulse emission times: with adiabatic faces every particle emitted
  before a sample time is counted at it, so the grid total at t_k is a
  binomial draw of the Gaussian time law truncated at t >= 0 (negative
  times redrawn);
* first-free-path truncation (max_collisions = 1): the same construction with
  the distance to the first film face or pore taken through the periodic
  lattice of pores (a 2-D walk over the unit cells the ray crosses);
* first-event truncation (max_events = 1) in the pored cell: each particle's
  mean contribution is |mu_z| Lambda (1 - exp(-d / Lambda)) for its distance d
  to the first boundary, and the quasi-Monte Carlo mean of that (numpy ray
  algebra, independent of the oracle) pins the emission law, the signs and
  the normalisation of the gradient source in pored geometries.
"""
import numpy as np
import pytest

import workloads as W


def _inside(prob, pos):
    g = prob["geometry"]
    x, y, z = pos
    if not (0.0 <= x <= g["L"] and 0.0 <= y <= g["pitch"] and 0.0 <= z <= g["pitch"]):
        return False
    dy, dz = y - 0.5 * g["pitch"], z - 0.5 * g["pitch"]
    return dy * dy + dz * dz >= g["radius"] ** 2


def _march(prob, pos, d, step):
    """Distance to the first exit of the solid unit cell, by marching + bisection."""
    t = 0.0
    while _inside(prob, pos + (t + step) * d):
        t += step
        if t > 10.0 * prob["geometry"]["L"]:
            return np.inf
    lo, hi = t, t + step
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if _inside(prob, pos + mid * d):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_first_boundary_against_marching(oracle):
    prob = W.porous_film(n_particles=1)
    g = prob["geometry"]
    rng = np.random.default_rng(3)
    n_done = 0
    kinds = set()
    while n_done < 300:
        pos = np.array([rng.uniform(0, g["L"]), rng.uniform(0, g["pitch"]), rng.uniform(0, g["pitch"])])
        if not _inside(prob, pos):
            continue
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t, kind = oracle.first_boundary(prob, pos, d)
        ref = _march(prob, pos, d, step=g["pitch"] / 200)
        assert t == pytest.approx(ref, rel=1e-9, abs=1e-9 * g["pitch"]), (pos, d, kind)
        kinds.add(kind)
        n_done += 1
    assert kinds == {1, 2, 3, 4, 5, 6, 7}


def test_zero_radius_porous_film_equals_film(oracle, analytic):
    L = 300e-9
    pin = analytic.kappa_film(W.SILICON_LIKE, L)
    p = W.porous_film(n_particles=2_000_000, radius=0.0, precision="fp64", max_events=1 << 16)
    r = oracle.run(p)
    assert r["periodic"] > 0
    assert abs(r["kappa"] - pin) < 4.0 * r["kappa_se"], (r["kappa"], pin, r["kappa_se"])


def test_pores_lower_conductivity(oracle, analytic):
    p = W.porous_film(n_particles=400_000, precision="fp64")
    r = oracle.run(p)
    film = analytic.kappa_film(W.SILICON_LIKE, 300e-9)
    porosity = np.pi * 0.3 ** 2
    assert 0.0 < r["kappa"] + 4 * r["kappa_se"]
    assert r["kappa"] + 4 * r["kappa_se"] < film * (1 - porosity)
    assert r["kappa_solid"] == pytest.approx(r["kappa"] / (1 - porosity), rel=1e-12)
    assert r["wall_hits"] > 0 and r["periodic"] > 0


def test_pulse_emission_in_solid(oracle):
    p = W.porous_pulse(n_particles=20_000, grid=(4, 8, 8), n_samples=10)
    st, _ = oracle.emit(p, 0, 20_000)
    g = p["geometry"]
    assert np.all(st[:, 0] == 1)
    assert np.all(st[:, 1] == g["L"]) and np.all(st[:, 4] < 0)
    yl = np.mod(st[:, 2], g["pitch"]) - 0.5 * g["pitch"]
    zl = np.mod(st[:, 3], g["pitch"]) - 0.5 * g["pitch"]
    assert np.all(yl * yl + zl * zl >= g["radius"] ** 2)
    assert np.all(st[:, 7] >= 0)
    t0 = st[:, 7]
    src = p["source"]
    assert abs(np.mean(t0) - src["t_center"]) < 5 * src["sigma_t"] / np.sqrt(t0.size) + 1e-13


def test_transient_energy_conservation(oracle):
    # all walls adiabatic, all particles positive: at every sample time the grid
    # holds exactly the particles already emitted (step VI only ends them at t_final)
    n = 3000
    p = W.porous_pulse(n_particles=n, grid=(4, 12, 12), n_samples=40, sample_dt=25e-12, t_final=1e-9)
    r = oracle.run(p, record_particles=True)
    grid = r["grid"]
    rec = r["particles_rec"]
    ts = (np.arange(40) + 0.5) * 25e-12
    emitted = np.array([(rec["t0"] <= t).sum() for t in ts])
    assert np.array_equal(grid.reshape(40, -1).sum(axis=1), emitted)
    assert np.all(grid >= 0)
    assert np.all(rec["fate"] == 3)


def _solid_fraction_yz(geo, ny, nz, sub=64):
    """Solid area fraction of each (y, z) grid column of the periodic domain."""
    Dy, Dz = geo["pitch"] * geo["cells_y"], geo["pitch"] * geo["cells_z"]
    frac = np.zeros((nz, ny))
    for iz in range(nz):
        for iy in range(ny):
            ys = (iy + (np.arange(sub) + 0.5) / sub) * Dy / ny
            zs = (iz + (np.arange(sub) + 0.5) / sub) * Dz / nz
            Y, Z = np.meshgrid(np.mod(ys, geo["pitch"]) - 0.5 * geo["pitch"],
                               np.mod(zs, geo["pitch"]) - 0.5 * geo["pitch"])
            frac[iz, iy] = np.mean(Y * Y + Z * Z >= geo["radius"] ** 2)
    return frac


def uniform_equilibrium_pvalues(grid, geo, times=(0, 10, 25, 49)):
    """p-values of 'counts are proportional to solid volume' at sample times."""
    from scipy import stats
    ns, nz, ny, nx = grid.shape
    w = np.repeat(_solid_fraction_yz(geo, ny, nz)[:, :, None], nx, axis=2)
    out = []
    for k in times:
        c = grid[k].astype(np.float64)
        e = c.sum() * w / w.sum()
        m = e > 0
        chi2 = (((c - e) ** 2)[m] / e[m]).sum()
        out.append(stats.chi2.sf(chi2, m.sum() - 1))
    return out


def test_initial_condition_energy_and_modes(oracle, analytic):
    n = 20_000
    p = W.porous_initial(n_particles=n, precision="fp64", x_range=(200e-9, 300e-9))
    r = oracle.run(p, record_particles=True)
    assert np.all(r["grid"].reshape(r["grid"].shape[0], -1).sum(axis=1) == n)  # exact, adiabatic walls
    rec = r["particles_rec"]
    assert np.all(rec["t0"] == 0.0) and np.all((rec["x0"] > 200e-9) & (rec["x0"] < 300e-9))
    area = (100e-9 ** 2 - np.pi * 30e-9 ** 2)
    assert r["E_eff"] == pytest.approx(r["C_tot"] * 1.0 * 100e-9 * area / n, rel=1e-12)
    # modes of the initial condition follow C_b (not C_b v_b)
    from scipy import stats
    _, v, tau, C = analytic.mode_table(W.SILICON_LIKE)
    u = (np.random.default_rng(4).integers(0, 2 ** 32, 400_000, dtype=np.uint64) + 0.5) / 2.0 ** 32
    modes = oracle.draw_modes(p, "initial", u)
    counts = np.bincount(modes, minlength=C.size)
    e = C / C.sum() * u.size
    keep = e > 20
    chi2 = ((counts[keep] - e[keep]) ** 2 / e[keep]).sum() + (counts[~keep].sum() - e[~keep].sum()) ** 2 / e[~keep].sum()
    assert stats.chi2.sf(chi2, keep.sum()) > 1e-4


@pytest.mark.parametrize("radius,g", [(0.0, 0.0), (30e-9, 0.0), (30e-9, 0.5)])
def test_uniform_initial_excess_stays_uniform(oracle, radius, g):
    # A uniform, isotropic excess with mode weights C_b is the linearized
    # equilibrium shape: free flights, Eq. 2 redraws and Lambertian walls must
    # all preserve it, so the counts stay proportional to the solid volume.
    # A direction law that depends only on the angle to the incoming direction
    # (anisotropic scattering, g != 0) maps an isotropic flux onto itself too.
    p = W.porous_initial(n_particles=200_000, precision="fp64", radius=radius,
                         material=dict(W.SILICON_LIKE, scatter_g=g))
    r = oracle.run(p)
    pv = uniform_equilibrium_pvalues(r["grid"], p["geometry"])
    assert min(pv) > 1e-4, pv


def test_ttr_layer_energy_is_conserved(oracle):
    # Thermoreflectance-like transient: the heated layer's energy only spreads
    # through the film (adiabatic faces), so every sample holds all particles,
    # and the solid-slab temperatures integrate to dT times the layer thickness.
    p = W.ttr_film(n_particles=50_000, precision="fp64", n_samples=40)
    r = oracle.run(p)
    counts = r["grid"].reshape(40, -1)  # nz = ny = 1: one count per x slab
    assert np.all(counts.sum(axis=1) == 50_000)
    L, nx = 300e-9, 30
    area = p["geometry"]["pitch"] ** 2
    Tx = counts * r["E_eff"] / (r["C_tot"] * area * L / nx)
    assert np.allclose(Tx.sum(axis=1) * L / nx, 1.0 * 30e-9, rtol=1e-12)
    # at the first sample (25 ps) the heat is still mostly in the top 60 nm
    assert Tx[0, -6:].sum() * L / nx > 0.8 * 30e-9


def map_symmetry_pvalues(o):
    """Chi-square p-values of the unit cell's mirror symmetries in the steady
    maps: T(y, z) = -T(y, pitch - z) = T(pitch - y, z) and q(y, z) =
    q(y, pitch - z) = q(pitch - y, z) (rows are z, columns y); each mirror
    pair of cells counted once."""
    from scipy import stats
    out = []
    for key, zsign in (("map_T", -1.0), ("map_q", 1.0)):
        v, se = o[key], o[key + "_se"]
        nz, ny = v.shape
        for axis, sgn in ((0, zsign), (1, 1.0)):
            flip, sflip = np.flip(v, axis), np.flip(se, axis)
            d = (v - sgn * flip) / np.sqrt(se ** 2 + sflip ** 2)
            half = d[: nz // 2, :] if axis == 0 else d[:, : ny // 2]
            half = half[np.isfinite(half)]
            out.append(stats.chi2.sf(np.sum(half ** 2), half.size))
    return out


@pytest.fixture(scope="module")
def pored_maps(oracle):
    return oracle.run(W.porous_film(n_particles=200_000, precision="fp64", map=(8, 8), n_batch=16))


def test_map_solid_fractions(oracle):
    pitch = 100e-9
    for ny, nz, r in ((8, 8, 30e-9), (7, 5, 45e-9)):
        o = oracle.run(W.porous_film(n_particles=64, precision="fp64", map=(ny, nz), radius=r))
        f = o["map_solid"]
        assert f.mean() == pytest.approx(1.0 - np.pi * (r / pitch) ** 2, abs=1e-13)
        np.testing.assert_allclose(f, f[::-1, :], atol=1e-13)
        np.testing.assert_allclose(f, f[:, ::-1], atol=1e-13)
        # a lattice of 400 x 400 points per cell, counted outside the disk
        m = 400
        for k in range(nz):
            z = (k + (np.arange(m) + 0.5) / m) * pitch / nz - 0.5 * pitch
            for j in range(ny):
                y = (j + (np.arange(m) + 0.5) / m) * pitch / ny - 0.5 * pitch
                frac = np.mean(y[None, :] ** 2 + z[:, None] ** 2 >= r * r)
                assert abs(frac - f[k, j]) < 3e-3, (ny, nz, k, j, frac, f[k, j])
        # cells wholly inside the pore hold no solid and report no value
        empty = f == 0.0
        assert np.all(np.isnan(o["map_T"][empty])) and np.all(np.isfinite(o["map_T"][~empty]))


def test_map_partitions_the_flux(pored_maps):
    # the z displacements over the map cells add up to the whole displacement
    o = pored_maps
    V = o["map_solid"] * (100e-9 / 8) ** 2 * 300e-9
    total = np.nansum(o["map_q"] * V)
    assert total == pytest.approx(o["flux"] * (100e-9) ** 2 * 300e-9, rel=1e-12)


def test_map_mirror_symmetries(pored_maps):
    o = pored_maps
    assert min(map_symmetry_pvalues(o)) > 1e-3, map_symmetry_pvalues(o)
    # and the maps are not flat: heat piles up below the pore (T > 0 at
    # z < pitch / 2 beside it) and the flux is lowest above and below it
    T, q = o["map_T"], o["map_q"]
    z = 5.0 * o["map_T_se"]
    assert T[1, 3] > z[1, 3] and T[6, 3] < -z[6, 3]
    assert q[0, 0] - q[0, 3] > 5.0 * np.hypot(o["map_q_se"][0, 0], o["map_q_se"][0, 3])


def test_map_of_film_is_flat(oracle, analytic):
    # no pores: no deviational temperature anywhere, the same flux everywhere
    from scipy import stats
    o = oracle.run(W.porous_film(n_particles=200_000, precision="fp64", map=(6, 6), radius=0.0, n_batch=16))
    np.testing.assert_allclose(o["map_solid"], 1.0, rtol=1e-13)
    zT = o["map_T"] / o["map_T_se"]
    assert stats.chi2.sf(np.sum(zT ** 2), zT.size) > 1e-3
    zq = (o["map_q"] - o["flux"]) / o["map_q_se"]
    assert stats.chi2.sf(np.sum(zq ** 2), zq.size - 1) > 1e-3
    assert abs(o["kappa"] - analytic.kappa_film(W.SILICON_LIKE, 300e-9)) < 4.0 * o["kappa_se"]


def first_event_pin_z(oracle, mat, radius, n=1_000_000, library=None, m=16):
    """z-score of the oracle's first-event pored-film conductivity against
    the quasi-Monte Carlo value (both errors combined)."""
    from oracle import analytic
    pin, pin_se = analytic.kappa_first_event_porous(mat, 300e-9, 100e-9, radius, m=m)
    prob = W.with_run(W.porous_film(n_particles=n, precision="fp64", material=mat, radius=radius), max_events=1)
    o = oracle.run(prob, library=library)
    return (o["kappa"] - pin) / np.hypot(o["kappa_se"], pin_se)


@pytest.mark.parametrize("lam,radius", [(2e-8, 30e-9), (2e-7, 30e-9), (5e-8, 45e-9), (1e-7, 0.0)])
def test_first_event_pored_film_against_quadrature(oracle, lam, radius):
    z = first_event_pin_z(oracle, dict(W.GRAY_UNIT, tau=lam, v=1.0), radius)
    assert abs(z) < 4.0, z


def test_first_event_silicon_pored_film_against_quadrature(oracle):
    z = first_event_pin_z(oracle, W.SILICON_LIKE, 30e-9, m=15)
    assert abs(z) < 4.0, z


def ballistic_spread_zmax(oracle, seed=5, library=None, n=200_000):
    """Largest |z| of the slab counts of a never-relaxing initial excess
    between specular faces against the folded free-streaming fractions."""
    from oracle import analytic
    L, v, dt, ns, nx = 300e-9, 1000.0, 20e-12, 30, 10
    p = W.porous_initial(n_particles=n, seed=seed, precision="fp64", material=dict(W.GRAY_UNIT, tau=1.0, v=v),
                         x_range=(200e-9, 260e-9), grid=(nx, 1, 1), n_samples=ns, sample_dt=dt, t_final=ns * dt,
                         radius=0.0)
    p["geometry"].update(wall_lo="specular", wall_hi="specular")
    o = oracle.run(p, library=library)
    frac = analytic.ballistic_slab_fractions(L, 200e-9, 260e-9, v, (np.arange(ns) + 0.5) * dt, nx)
    c = o["grid"].reshape(ns, nx).astype(float)
    e = frac * n
    sd = np.sqrt(np.maximum(e * (1.0 - frac), 1e-300))
    z = np.where(e > 5, (c - e) / sd, 0.0)
    # slabs the kinematics leave empty must stay empty
    assert np.all(c[frac == 0] == 0)
    return float(np.max(np.abs(z)))


def test_ballistic_spreading_between_specular_faces(oracle):
    assert ballistic_spread_zmax(oracle) < 5.0


def pulse_totals_zmax(oracle, library=None, n=200_000, precision="fp64", run=None):
    """Largest |z| of the pulse's per-sample grid totals against N F(t_k),
    F the Gaussian CDF of the emission time conditioned on t >= 0.  ``run``
    replaces the oracle (the GPU tests pass the library's simulate)."""
    from scipy.stats import norm
    tc, st, dt, ns = 50e-12, 100e-12, 10e-12, 40
    p = W.porous_pulse(n_particles=n, precision=precision, material=dict(W.GRAY_UNIT, tau=1e-10, v=1000.0),
                       grid=(4, 6, 6), n_samples=ns, sample_dt=dt, t_final=ns * dt)
    p["source"].update(t_center=tc, sigma_t=st)
    r = run(p) if run is not None else oracle.run(p, library=library)
    tot = r["grid"].reshape(ns, -1).sum(axis=1).astype(float)
    tk = (np.arange(ns) + 0.5) * dt
    p0 = norm.cdf(-tc / st)
    F = (norm.cdf((tk - tc) / st) - p0) / (1.0 - p0)
    sd = np.sqrt(n * F * (1.0 - F))
    return float(np.max(np.abs(tot - n * F) / sd))


def test_pulse_emission_times(oracle):
    assert pulse_totals_zmax(oracle) < 5.0


def pulse_lateral_pvalues(oracle, library=None, n=100_000):
    """KS p-values of the pulse's emitted lateral radius (r^2 / 2 sigma^2
    against Exp(1), minimum-image distance in the periodic domain) and of its
    direction cosine into the film (mu_x^2 against U(0, 1)), without pores."""
    from scipy import stats
    p = W.porous_pulse(n_particles=n, grid=(4, 8, 8), n_samples=10, radius=0.0)
    st, _ = oracle.emit(p, 0, n, library=library)
    g, src = p["geometry"], p["source"]
    Dy, Dz = g["pitch"] * g["cells_y"], g["pitch"] * g["cells_z"]
    dy = np.mod(st[:, 2] - src["y0"] + 0.5 * Dy, Dy) - 0.5 * Dy
    dz = np.mod(st[:, 3] - src["z0"] + 0.5 * Dz, Dz) - 0.5 * Dz
    r2 = (dy * dy + dz * dz) / (2.0 * src["sigma_x"] ** 2)
    return stats.kstest(r2, "expon").pvalue, stats.kstest(st[:, 4] ** 2, "uniform").pvalue


def test_pulse_lateral_law_and_directions(oracle):
    p_r, p_mu = pulse_lateral_pvalues(oracle)
    assert p_r > 1e-3 and p_mu > 1e-3, (p_r, p_mu)


def free_path_pin_z(oracle, mat, radius, n=1_000_000, library=None, m=16):
    """z-score of the oracle's first-free-path pored-film conductivity against
    the quasi-Monte Carlo value through the periodic lattice of pores."""
    from oracle import analytic
    pin, pin_se = analytic.kappa_free_path_porous(mat, 300e-9, 100e-9, radius, m=m)
    prob = W.with_run(W.porous_film(n_particles=n, precision="fp64", material=mat, radius=radius), max_collisions=1)
    o = oracle.run(prob, library=library)
    return (o["kappa"] - pin) / np.hypot(o["kappa_se"], pin_se)


@pytest.mark.parametrize("lam,radius", [(2e-8, 30e-9), (2e-7, 30e-9), (5e-8, 45e-9)])
def test_first_free_path_pored_film_against_quadrature(oracle, lam, radius):
    z = free_path_pin_z(oracle, dict(W.GRAY_UNIT, tau=lam, v=1.0), radius)
    assert abs(z) < 4.0, z


def test_first_free_path_silicon_pored_film_against_quadrature(oracle):
    z = free_path_pin_z(oracle, W.SILICON_LIKE, 30e-9, m=15)
    assert abs(z) < 4.0, z
