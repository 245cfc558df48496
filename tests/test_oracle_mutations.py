"""The pins must be able to fail: plant one plausible mistake at a time in a
copy of the oracle's C source (never in the oracle itself), compile it, and
check that the pin guarding that step rejects it while the unmodified oracle
passes the same check."""
import numpy as np
import pytest

import workloads as W


def _psi_pin_ok(oracle, analytic, library):
    n = 2_000_000
    r = oracle.run(W.gray_slab(n_particles=n, kn=1.0, n_bins=0), library=library)
    pin = analytic.slab_solution(1.0, n_bins=50, M=100)["psi"]
    return abs(r["psi"] - pin) < 4.0 * np.sqrt(pin * (1 - pin) / n)


def _film_pin_ok(oracle, analytic, library):
    r = oracle.run(W.silicon_film(n_particles=400_000, precision="fp64", max_events=1), library=library)
    return abs(r["kappa"] - analytic.kappa_film(W.SILICON_LIKE, 100e-9)) < 4.0 * r["kappa_se"]


def _bulk_pin_ok(oracle, analytic, library):
    mat = dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0)
    r = oracle.run(W.bulk(n_particles=400_000, material=mat, max_events=8), library=library)
    return abs(r["kappa"] - 7.0 * 9.0 * 2.5 / 3.0) < 4.0 * r["kappa_se"]


def _nongray_pin_ok(oracle, analytic, library):
    mat = dict(W.SILICON_LIKE, n_bins=10)
    _, v, tau, C = analytic.mode_table(mat)
    pin = analytic.slab_multimode_psi(v * tau, C * v, C / tau, 100e-9, M=60)
    p = W.gray_slab(n_particles=400_000, n_bins=0)
    p["material"] = mat
    p["geometry"]["L"] = 100e-9
    r = oracle.run(p, library=library)
    return abs(r["psi"] - pin) < 4.0 * r["psi_se"]


def _uniform_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import uniform_equilibrium_pvalues
    p = W.porous_initial(n_particles=200_000, precision="fp64", radius=0.0)
    r = oracle.run(p, library=library)
    return min(uniform_equilibrium_pvalues(r["grid"], p["geometry"])) > 1e-4


def _pore_uniform_pin_ok(oracle, analytic, library):
    # A uniform isotropic excess in a pored cell stays uniform (counts in
    # proportion to the solid volume) and whole (adiabatic walls) only if the
    # pore wall re-emits with the cosine law about the normal pointing into
    # the solid.  (Segment cap 4096: a law that sends particles into the pore
    # pins them to the wall in zero-length segments, which the cap ends.)
    p = W.porous_initial(n_particles=200_000, precision="fp64", radius=30e-9, max_events=4096)
    r = oracle.run(p, library=library)
    totals = r["grid"].reshape(r["grid"].shape[0], -1).sum(axis=1)
    if not np.all(totals == 200_000):
        return False
    from tests.test_oracle_porous import uniform_equilibrium_pvalues
    return min(uniform_equilibrium_pvalues(r["grid"], p["geometry"])) > 1e-4


def _specular_pin_ok(oracle, analytic, library):
    r = oracle.run(W.silicon_film(n_particles=1_000_000, precision="fp64", specularity=0.25), library=library)
    return abs(r["kappa"] - analytic.kappa_film(W.SILICON_LIKE, 100e-9, 0.25)) < 4.0 * r["kappa_se"]


def _first_path_pin_ok(oracle, analytic, library):
    r = oracle.run(W.with_run(W.silicon_film(n_particles=400_000, precision="fp64"), max_collisions=1),
                   library=library)
    # (the film is symmetric enough that stopping at the first relaxation is
    # also exact, so the one-segment-per-particle count is what tells them apart)
    return (abs(r["kappa"] - analytic.kappa_film(W.SILICON_LIKE, 100e-9)) < 4.0 * r["kappa_se"]
            and r["segments"] == r["particles"])


def _aniso_split_pin_ok(oracle, analytic, library):
    g = 0.6
    p = W.bulk(n_particles=300_000, material=dict(W.GRAY_UNIT, scatter_g=g), dTdz=-1.0)
    p["run"]["n_hj"] = 4
    r = oracle.run(p, library=library)
    H, se = r["H"], r["H_se"]
    return all(abs(H[j] / H[0] - g ** j) < 4.0 * abs(H[j] / H[0]) * np.hypot(se[j] / H[j], se[0] / H[0]) + 1e-12
               for j in (1, 2))


def _aniso_bulk_pin_ok(oracle, analytic, library):
    mat = dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0, scatter_g=0.5)
    r = oracle.run(W.bulk(n_particles=200_000, material=mat), library=library)
    return abs(r["kappa"] - 105.0) < 4.0 * r["kappa_se"]


def _flight_shape_pin_ok(oracle, analytic, library):
    lam, n = 7.5, 400_000
    r = oracle.run(W.bulk(n_particles=n, material=dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0), max_events=1),
                   library=library)
    return abs(r["sum_sL2"] / n - lam ** 2) < 4.0 * np.sqrt(7.0 / n) * lam ** 2


def _map_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import map_symmetry_pvalues
    r = oracle.run(W.porous_film(n_particles=200_000, precision="fp64", map=(8, 8), n_batch=16), library=library)
    return min(map_symmetry_pvalues(r)) > 1e-3


def _first_event_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import first_event_pin_z
    return abs(first_event_pin_z(oracle, dict(W.GRAY_UNIT, tau=5e-8, v=1.0), 45e-9, n=400_000, library=library)) < 4.0


def _ballistic_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import ballistic_spread_zmax
    try:
        return ballistic_spread_zmax(oracle, library=library, n=100_000) < 5.0
    except AssertionError:
        return False


def _pulse_time_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import pulse_totals_zmax
    return pulse_totals_zmax(oracle, library=library, n=100_000) < 5.0


def _pulse_lateral_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import pulse_lateral_pvalues
    return min(pulse_lateral_pvalues(oracle, library=library)) > 1e-3


def _film_profile_pin_ok(oracle, analytic, library):
    from tests.test_oracle_transport import film_profile_pvalues
    try:
        return min(film_profile_pvalues(oracle, analytic, library=library)) > 1e-3
    except AssertionError:  # the bins no longer partition the flux
        return False


def _free_path_pin_ok(oracle, analytic, library):
    from tests.test_oracle_porous import free_path_pin_z
    return abs(free_path_pin_z(oracle, dict(W.GRAY_UNIT, tau=2e-7, v=1.0), 30e-9, n=400_000, library=library)) < 4.0


MUTATIONS = [
    ("diffuse wall re-emission not Lambertian", "dir_axis(0, sqrt(u[2]), u[3], &s.ox, &s.oy, &s.oz);",
     "dir_axis(0, u[2], u[3], &s.ox, &s.oy, &s.oz);", _uniform_pin_ok),
    # (name, original text, planted mistake, pin that must catch it)
    # (a law that only folds directions into one z hemisphere is invisible to
    # every steady estimator here: the gradient source emits equal numbers of
    # each sign and a hemisphere projects onto x like the sphere; the planted
    # law below is genuinely anisotropic)
    ("scattering not isotropic",
     "s.mode = draw_mode(m->cdf_scat, m->n, u[1]);\n            dir_axis(2, 2.0 * u[2] - 1.0, u[3]",
     "s.mode = draw_mode(m->cdf_scat, m->n, u[1]);\n            dir_axis(2, 2.0 * u[2] * u[2] - 1.0, u[3]",
     _psi_pin_ok),
    ("bulk flight with wrong mean free path", "double dist = m->Lambda[s.mode] * -log(u[0]);",
     "double dist = 0.5 * m->Lambda[s.mode] * -log(u[0]);", _bulk_pin_ok),
    ("wall emission not cosine weighted", "int lo = u[0] * (wlo + whi) < wlo;\n        double mu = sqrt(u[2]);",
     "int lo = u[0] * (wlo + whi) < wlo;\n        double mu = u[2];", _psi_pin_ok),
    ("Eq. 2 redraw from the emission law", "s.mode = draw_mode(m->cdf_scat", "s.mode = draw_mode(m->cdf_emit",
     _nongray_pin_ok),
    ("gradient-source sign flipped", "(p->dTdz > 0.0 ? -1.0 : 1.0)", "(p->dTdz > 0.0 ? 1.0 : -1.0)", _film_pin_ok),
    ("flight drawn with the wrong mean free path", "double dist = m->Lambda[s.mode] * -log(u[0]);",
     "double dist = m->tau[s.mode] * -log(u[0]);", _film_pin_ok),
    ("partial wall specular with probability 1 - p", "wall_type = u[1] < spec ? ORC_WALL_SPECULAR",
     "wall_type = u[1] >= spec ? ORC_WALL_SPECULAR", _specular_pin_ok),
    ("specular reflection also flips the in-plane direction", "if (wall_type == ORC_WALL_SPECULAR) s.ox = -s.ox;",
     "if (wall_type == ORC_WALL_SPECULAR) { s.ox = -s.ox; s.oz = -s.oz; }", _specular_pin_ok),
    ("first-free-path cap counts only relaxations", "n_scat + n_wall >= p->max_collisions",
     "n_scat >= p->max_collisions", _first_path_pin_ok),
    ("anisotropic law about the z axis, not the incoming direction",
     "hg_direction(p->scatter_g, u[2], u[3], in_x, in_y, in_z,", "hg_direction(p->scatter_g, u[2], u[3], 0.0, 0.0, 1.0,",
     _aniso_split_pin_ok),
    ("anisotropic cosine with the wrong sign", "double mu = (1.0 + g * g - q * q) / (2.0 * g);",
     "double mu = -(1.0 + g * g - q * q) / (2.0 * g);", _aniso_bulk_pin_ok),
    ("flight length uniform on [0, 2 Lambda] (right mean, wrong law)", "double dist = m->Lambda[s.mode] * -log(u[0]);",
     "double dist = m->Lambda[s.mode] * 2.0 * u[0];", _flight_shape_pin_ok),
    ("density of states missing a factor k", "double dos = k * k / (2.0 * ORC_PI * ORC_PI * vg);",
     "double dos = k / (2.0 * ORC_PI * ORC_PI * vg);", _film_pin_ok),
    ("steady map cells indexed (y, z) instead of (z, y)",
     "T[(size_t)k * ny + j] += s->sign * ((b - a) / vg);\n            q[(size_t)k * ny + j]",
     "T[(size_t)j * nz + k] += s->sign * ((b - a) / vg);\n            q[(size_t)j * nz + k]", _map_pin_ok),
    ("steady map time tallied without the particle's sign", "T[(size_t)k * ny + j] += s->sign * ((b - a) / vg);",
     "T[(size_t)k * ny + j] += (b - a) / vg;", _map_pin_ok),
    ("sample positions interpolated from t = 0 instead of the segment start",
     "double d = vg * (ts - t_a);", "double d = vg * ts;", _ballistic_pin_ok),
    ("pulse times below zero moved to zero instead of redrawn", "if (t0 >= 0.0) { s->t = t0; break; }",
     "if (t0 < 0.0) t0 = 0.0;\n            { s->t = t0; break; }", _pulse_time_pin_ok),
    ("pulse lateral radius with a Gaussian variance halved",
     "double r = p->pulse_sigma_x * sqrt(-2.0 * log(v[0]));", "double r = p->pulse_sigma_x * sqrt(-log(v[0]));",
     _pulse_lateral_pin_ok),
    ("in-plane flux by depth without the 1/|ox| of the path's slope", "q[k] += sign * (len * oz / fabs(ox));",
     "q[k] += sign * (len * oz);", _film_profile_pin_ok),
    ("first-free-path cap also counting crossings of periodic unit-cell faces",
     "n_scat + n_wall >= p->max_collisions", "n_scat + n_wall + n_per >= p->max_collisions", _free_path_pin_ok),
    ("pore-wall re-emission uniform in the cosine (not Lambertian)",
     "double mu = sqrt(u[2]);\n                        double st = sqrt(fmax(0.0, 1.0 - mu * mu));\n"
     "                        double phi = ORC_TWO_PI * u[3];",
     "double mu = u[2];\n                        double st = sqrt(fmax(0.0, 1.0 - mu * mu));\n"
     "                        double phi = ORC_TWO_PI * u[3];", _pore_uniform_pin_ok),
    ("pore-wall cosine law about the normal pointing into the pore",
     "s.oy = mu * ny - st * sn * nz;\n                        s.oz = mu * nz + st * sn * ny;",
     "s.oy = -mu * ny - st * sn * nz;\n                        s.oz = -mu * nz + st * sn * ny;",
     _pore_uniform_pin_ok),
    ("gradient-source positions not restricted to the solid",
     "                s->cy = cy; s->cz = cz; s->y = yl; s->z = zl;\n                if (!in_pore(p, yl, zl)) break;",
     "                s->cy = cy; s->cz = cz; s->y = yl; s->z = zl;\n                break;", _first_event_pin_ok),
]


@pytest.mark.parametrize("name,orig,bad,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(oracle, analytic, tmp_path, name, orig, bad, pin):
    text = oracle.source_text()
    assert text.count(orig) == 1, name
    assert pin(oracle, analytic, None), "the unmodified oracle must pass " + pin.__name__
    lib = oracle.compile_variant(text.replace(orig, bad), str(tmp_path / "mutant.so"))
    assert not pin(oracle, analytic, lib), f"pin {pin.__name__} missed: {name}"
