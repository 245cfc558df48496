"""GPU parity for the wall-law variants and the first-free-path truncation.

* partially specular walls (specular with probability p, diffuse otherwise):
  FP64 single-mode runs follow the oracle particle by particle (the choice is
  made from the same uniform on both sides); FP32 silicon films against the
  Fuchs-Sondheimer factor with specularity p;
* first-free-path truncation (stop at the first relaxation or wall hit,
  periodic faces not counted): exact for the diffuse film, an overestimate
  for the pored film, and the same as the oracle's.
"""
import numpy as np
import pytest

import workloads as W
from tests.test_gpu_parity import _same_particles, _z

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def test_gray_film_partial_walls_per_particle(P, oracle):
    prob = W.silicon_film(n_particles=4000, thickness=0.7, material=dict(W.GRAY_UNIT), precision="fp64",
                          max_scatter=12, max_events=200, dTdz=-1.0)
    prob["geometry"].update(wall_lo="partial", wall_hi="partial", spec_lo=0.3, spec_hi=0.8)
    g = P.simulate(prob, record_particles=True)
    o = oracle.run(prob, record_particles=True)
    _same_particles(g["particles_rec"], o["particles_rec"])
    assert g["wall_hits"] == o["wall_hits"] > 0


def test_gray_slab_partial_walls_per_particle(P, oracle):
    prob = W.gray_slab(n_particles=3000, n_bins=0, walls=("partial", "black"), dT=(1.0, -0.5))
    prob["geometry"]["spec_lo"] = 0.6
    prob["run"]["max_events"] = 500
    g = P.simulate(prob, record_particles=True)
    o = oracle.run(prob, record_particles=True)
    _same_particles(g["particles_rec"], o["particles_rec"])


def test_gray_porous_partial_pores_per_particle(P, oracle):
    prob = W.porous_film(n_particles=3000, precision="fp64", material=dict(W.GRAY_UNIT, tau=2e-8, v=1.0),
                         max_events=300, max_scatter=20)
    prob["geometry"].update(pore_wall="partial", spec_pore=0.5, wall_lo="partial", spec_lo=0.2)
    g = P.simulate(prob, record_particles=True)
    o = oracle.run(prob, record_particles=True)
    _same_particles(g["particles_rec"], o["particles_rec"], atol=2e-8 * 1e-6)


@pytest.mark.parametrize("p", [0.25, 0.75])
def test_partially_specular_silicon_film_fp32(P, oracle, analytic, p):
    pin = analytic.kappa_film(W.SILICON_LIKE, 100e-9, p)
    g = P.simulate(W.silicon_film(n_particles=40_000_000, specularity=p))
    assert abs(g["kappa"] - pin) < 3.0 * g["kappa_se"], (g["kappa"], pin, g["kappa_se"])
    o = oracle.run(W.silicon_film(n_particles=500_000, precision="fp64", specularity=p))
    assert _z(g, o, "kappa") < 3.0


def test_first_free_path_film_exact(P, analytic):
    pin = analytic.kappa_film(W.SILICON_LIKE, 100e-9)
    g = P.simulate(W.with_run(W.silicon_film(n_particles=20_000_000), max_collisions=1))
    assert g["segments"] == g["particles"] == g["truncated"]
    assert abs(g["kappa"] - pin) < 3.0 * g["kappa_se"], (g["kappa"], pin)


def test_first_free_path_overestimates_pored_film(P, oracle):
    full = P.simulate(W.porous_film(n_particles=20_000_000))
    first = P.simulate(W.with_run(W.porous_film(n_particles=20_000_000), max_collisions=1))
    print(f"\npored film: kappa {full['kappa']:.3f} +- {full['kappa_se']:.3f}; first free path only "
          f"{first['kappa']:.3f} +- {first['kappa_se']:.3f} ({100 * (first['kappa'] / full['kappa'] - 1):+.0f} %)")
    assert first["scatters"] + first["wall_hits"] == first["particles"] and first["periodic"] > 0
    assert first["kappa"] - full["kappa"] > 5.0 * np.hypot(first["kappa_se"], full["kappa_se"])
    o = oracle.run(W.with_run(W.porous_film(n_particles=400_000, precision="fp64"), max_collisions=1))
    assert _z(first, o, "kappa") < 3.0


def test_first_free_path_pored_film_against_quadrature(P, analytic):
    # config-2 steady at full size, max_collisions = 1, FP32: against the
    # quasi-Monte Carlo first-free-path conductivity through the periodic
    # lattice of pores (numpy ray algebra)
    pin, pin_se = analytic.kappa_free_path_porous(W.SILICON_LIKE, 300e-9, 100e-9, 30e-9, m=16)
    g = P.simulate(W.with_run(W.porous_film(n_particles=100_000_000), max_collisions=1), arrays=False)
    z = (g["kappa"] - pin) / np.hypot(g["kappa_se"], pin_se)
    print(f"\nfirst free path, pored film: GPU {g['kappa']:.4f} +- {g['kappa_se']:.4f}, "
          f"quadrature {pin:.4f} +- {pin_se:.4f}")
    assert abs(z) < 4.0, z


def test_invalid_specularity_rejected(P):
    prob = W.silicon_film(n_particles=10, specularity=1.5)
    with pytest.raises(Exception):
        P.simulate(prob)


def test_collision_cap_per_particle(P, oracle):
    # the cap is folded into the segment cap for films (every segment ends in a
    # collision there) and checked per segment in pored films: both report the
    # collision-cap fate exactly where the oracle does
    film = W.silicon_film(n_particles=3000, thickness=0.7, material=dict(W.GRAY_UNIT), precision="fp64",
                          max_scatter=12, max_events=200, dTdz=-1.0)
    pores = W.porous_film(n_particles=3000, precision="fp64", material=dict(W.GRAY_UNIT, tau=2e-8, v=1.0),
                          max_events=300, max_scatter=20)
    for prob, atol in ((film, 1e-12), (pores, 2e-8 * 1e-6)):
        for cap in (1, 3, 250):
            p = W.with_run(prob, max_collisions=cap)
            g = P.simulate(p, record_particles=True)
            o = oracle.run(p, record_particles=True)
            _same_particles(g["particles_rec"], o["particles_rec"], atol=atol)
            if cap < 10:
                assert 4 in set(np.unique(g["particles_rec"]["fate"]).tolist()), cap
