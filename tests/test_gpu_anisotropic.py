"""GPU parity for anisotropic relaxation events (Henyey-Greenstein direction
law of mean cosine g about the incoming direction; the paper's isotropic
redraw is g = 0).

* FP64 single-mode runs follow the oracle particle by particle (same
  uniforms, same inverted CDF, same orthonormal frame);
* FP32 runs against the closed forms: bulk conductivity, and the flux split
  by relaxation index, which is geometric with ratio g in a gray bulk;
* an isotropic, uniform excess stays uniform (the law maps an isotropic flux
  onto itself).
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


@pytest.mark.parametrize("g", [0.6, -0.4])
def test_gray_film_anisotropic_per_particle(P, oracle, g):
    prob = W.silicon_film(n_particles=4000, thickness=0.7, material=dict(W.GRAY_UNIT, scatter_g=g),
                          precision="fp64", max_scatter=12, max_events=200, dTdz=-1.0, n_hj=8)
    g_ = P.simulate(prob, record_particles=True)
    o = oracle.run(prob, record_particles=True)
    _same_particles(g_["particles_rec"], o["particles_rec"], atol=1e-10)


def test_gray_porous_anisotropic_per_particle(P, oracle):
    prob = W.porous_film(n_particles=3000, precision="fp64", max_events=300, max_scatter=20,
                         material=dict(W.GRAY_UNIT, tau=2e-8, v=1.0, scatter_g=0.5))
    g = P.simulate(prob, record_particles=True)
    o = oracle.run(prob, record_particles=True)
    _same_particles(g["particles_rec"], o["particles_rec"], atol=2e-8 * 1e-6)


def test_anisotropic_bulk_fp32_against_closed_form(P, oracle, analytic):
    gray = dict(W.GRAY_UNIT, tau=2.5, v=3.0, C=7.0, scatter_g=0.5)
    r = P.simulate(W.bulk(n_particles=20_000_000, material=gray, precision="fp32"))
    assert abs(r["kappa"] - 105.0) < 3.0 * r["kappa_se"], (r["kappa"], r["kappa_se"])
    si = dict(W.SILICON_LIKE, scatter_g=0.4)
    pin = analytic.kappa_bulk_anisotropic(si, 0.4)
    r = P.simulate(W.bulk(n_particles=50_000_000, material=si, precision="fp32"))
    assert abs(r["kappa"] - pin) < 3.0 * r["kappa_se"], (r["kappa"], pin, r["kappa_se"])
    o = oracle.run(W.bulk(n_particles=1_000_000, material=si, precision="fp64"))
    assert _z(r, o, "kappa") < 3.0


def test_anisotropic_flux_split_fp32(P):
    g = 0.6
    p = W.bulk(n_particles=20_000_000, material=dict(W.GRAY_UNIT, scatter_g=g), dTdz=-1.0, precision="fp32")
    p["run"]["n_hj"] = 8
    r = P.simulate(p)
    H, se = r["H"], r["H_se"]
    for j in range(1, 7):
        ratio = H[j] / H[0]
        err = abs(ratio) * np.hypot(se[j] / H[j], se[0] / H[0])
        assert abs(ratio - g ** j) < 3.0 * err, (j, ratio, g ** j, err)


def test_anisotropic_uniform_excess_stays_uniform(P):
    from tests.test_oracle_porous import uniform_equilibrium_pvalues
    n = 2_000_000
    prob = W.porous_initial(n_particles=n, precision="fp32", material=dict(W.SILICON_LIKE, scatter_g=0.5))
    g = P.simulate(prob)
    assert np.all(g["grid"].reshape(g["grid"].shape[0], -1).sum(axis=1) == n)
    assert min(uniform_equilibrium_pvalues(g["grid"], prob["geometry"])) > 1e-4


def test_invalid_anisotropy_rejected(P):
    with pytest.raises(P.LeMcError):
        P.simulate(W.bulk(n_particles=10, material=dict(W.GRAY_UNIT, scatter_g=1.0)))
