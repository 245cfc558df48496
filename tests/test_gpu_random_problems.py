"""Seeded random problems, GPU (FP64, single-mode gray materials) against the
oracle.

Slabs, films, bulk media, pored films (with and without maps), surface
pulses and initial excesses, with random sizes, wall laws, partial
specularities, anisotropy, caps and sampling windows.  Every run traces all
its particles with no device flag set.  Where the dynamics do not amplify
rounding, histories agree particle by particle.  Specular pores, or mean free
paths far above the pore radius, make the pored cell a dispersing billiard:
the last-bit differences between the GPU's fused multiply-adds and libm and
the oracle's separately rounded arithmetic then grow from reflection to
reflection until some histories part.  There the runs must agree in
distribution instead: identical transient sample totals (emission does not
depend on the history), conductivities within 4 sigma.
"""
import copy

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

WALLS = ["black", "diffuse", "specular", "partial"]
PORE = ["diffuse", "specular", "partial"]


def random_problem(rng):
    kind = str(rng.choice(["slab", "film", "porous", "pulse", "initial", "bulk"]))
    tau = float(10 ** rng.uniform(-11, -9)); v = float(10 ** rng.uniform(2.5, 3.7))
    g = float(rng.choice([0.0, 0.0, 0.3, -0.5, 0.8]))
    mat = dict(W.GRAY_UNIT, tau=tau, v=v, scatter_g=g)
    n = int(rng.integers(200, 3000))
    lam = tau * v
    if kind == "slab":
        walls = (str(rng.choice(WALLS)), str(rng.choice(WALLS)))
        if "black" not in walls:
            walls = ("black", walls[1])
        p = W.gray_slab(n_particles=n, kn=float(10 ** rng.uniform(-1, 1)), n_bins=int(rng.choice([0, 7])), walls=walls)
        p["material"]["scatter_g"] = g
        p["run"]["max_events"] = int(rng.choice([50, 4096]))
    elif kind == "film":
        walls = (str(rng.choice(WALLS[1:])), str(rng.choice(WALLS[1:])))
        L = float(lam * 10 ** rng.uniform(-1, 1))
        p = W.silicon_film(n_particles=n, thickness=L, material=mat, precision="fp64", walls=walls,
                           max_scatter=int(rng.choice([0, 5, 40])), max_events=int(rng.choice([1, 50, 4096])),
                           n_hj=int(rng.choice([0, 6])))
    elif kind == "bulk":
        p = W.bulk(n_particles=n, material=mat, max_scatter=int(rng.choice([5, 40])), max_events=int(rng.choice([50, 400])))
    else:
        pitch = float(lam * 10 ** rng.uniform(-0.5, 1)); radius = float(pitch * rng.uniform(0, 0.45))
        L = float(pitch * 10 ** rng.uniform(-0.3, 0.7))
        if kind == "porous":
            p = W.porous_film(n_particles=n, precision="fp64", material=mat, thickness=L, pitch=pitch, radius=radius,
                              max_scatter=int(rng.choice([0, 5, 40])), max_events=int(rng.choice([1, 50, 400])),
                              map=(int(rng.integers(1, 9)), int(rng.integers(1, 9))) if rng.random() < 0.5 else None)
        elif kind == "pulse":
            ns = int(rng.integers(1, 30)); dt = float(lam / v * rng.uniform(0.2, 3))
            p = W.porous_pulse(n_particles=n, precision="fp64", material=mat, thickness=L, pitch=pitch, radius=radius,
                               grid=(int(rng.integers(1, 6)), int(rng.integers(1, 6)), int(rng.integers(1, 6))),
                               n_samples=ns, sample_dt=dt, t_final=float(dt * ns * rng.choice([1.0, 1.0, 3.0])),
                               cells=(int(rng.integers(1, 4)), int(rng.integers(1, 4))), max_events=400)
            p["source"]["sigma_x"] = float(pitch * rng.uniform(0.2, 2)); p["source"]["sigma_t"] = float(dt * rng.uniform(0.5, 5))
            p["source"]["t_center"] = float(dt * rng.uniform(0, 5))
        else:
            ns = int(rng.integers(1, 30)); dt = float(lam / v * rng.uniform(0.2, 3))
            lo = float(L * rng.uniform(0, 0.5)); hi = float(lo + (L - lo) * rng.uniform(0.1, 1))
            p = W.porous_initial(n_particles=n, precision="fp64", material=mat, thickness=L, pitch=pitch, radius=radius,
                                 grid=(int(rng.integers(1, 6)), int(rng.integers(1, 6)), int(rng.integers(1, 6))),
                                 n_samples=ns, sample_dt=dt, t_final=float(dt * ns * rng.choice([1.0, 3.0])),
                                 x_range=(lo, hi), max_events=400)
        p["geometry"]["wall_lo"] = str(rng.choice(WALLS[1:])); p["geometry"]["wall_hi"] = str(rng.choice(WALLS[1:]))
        p["geometry"]["pore_wall"] = str(rng.choice(PORE))
    geo = p["geometry"]
    for k in ("spec_lo", "spec_hi", "spec_pore"):
        geo[k] = float(rng.uniform(0, 1))
    if rng.random() < 0.3:
        p["run"]["max_collisions"] = int(rng.choice([1, 3]))
    p["run"]["seed"] = int(rng.integers(1, 2**62))
    return kind, p




@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def _diverged(g, o, p):
    gr, orr = g["particles_rec"], o["particles_rec"]
    for f in ("sign", "fate", "n_seg", "n_scat", "n_wall", "n_periodic", "mode0"):
        if not np.array_equal(gr[f], orr[f]):
            return True
    scale = max(abs(p["geometry"].get("L", 1.0)), p["material"].get("tau", 1) * p["material"].get("v", 1))
    if len(gr) and np.max(np.abs(gr["L_axis"] - orr["L_axis"])) > 1e-6 * scale:
        return True
    return "grid" in g and not np.array_equal(g["grid"].astype(np.int64), o["grid"])


@pytest.mark.parametrize("seed", [7, 11, 2012])
def test_random_problems_against_oracle(P, oracle, seed):
    rng = np.random.default_rng(seed)
    exact = 0
    for i in range(40):
        kind, p = random_problem(rng)
        try:
            g = P.simulate(p, record_particles=True)
        except P.LeMcError:
            with pytest.raises(ValueError):
                oracle.run(p)
            continue
        o = oracle.run(p, record_particles=True)
        assert g["device_flags"] == 0 and g["particles"] == p["run"]["n_particles"], (seed, i, kind)
        if not _diverged(g, o, p):
            exact += 1
            continue
        q = copy.deepcopy(p)
        q["run"]["n_particles"] = 20_000
        gq, oq = P.simulate(q), oracle.run(q)
        if "grid" in gq:
            tg = gq["grid"].reshape(gq["grid"].shape[0], -1).sum(axis=1)
            to = oq["grid"].reshape(oq["grid"].shape[0], -1).sum(axis=1)
            assert np.array_equal(tg, to), (seed, i, kind)
        else:
            key = "kappa" if q["source"]["kind"] == "gradient" else "psi"
            z = abs(gq[key] - oq[key]) / np.hypot(gq[key + "_se"], oq[key + "_se"])
            assert z < 4.0, (seed, i, kind, z)
    assert exact >= 25, exact
