"""Seeded synthetic workloads shared by the tests, the benchmark and smoke().

This module only holds problem *parameters* (plain dicts of numbers and
strings) and the seeded draws of instance parameters.  It contains none of the
method's arithmetic: material tables, sources, tracing and estimators are
computed independently by the oracle (``oracle/``) and by the CUDA library
(``paper_1206_3316_gb300/``), each from these parameters.

A problem is a dict with four parts::

    {"material": {...}, "geometry": {...}, "source": {...}, "run": {...}}

Units are SI (m, s, K, J) except for the non-dimensional gray slab, where the
group velocity, relaxation time, heat capacity and thickness are all 1.

The paper's applications use material data and geometries (its Refs. 11-12
and the unit cell of its Fig. 2) that are not available; the workloads below
are synthetic stand-ins with the shapes and scales of those problems.
"""
from __future__ import annotations

import copy
import math

import numpy as np

# Isotropic quadratic dispersion omega(k) = c1 k + c2 k^2 with silicon-like
# coefficients: one LA branch and the two degenerate TA branches (degeneracy 2),
# k up to 2 pi / 5.43 A, 1000 frequency bins per branch; relaxation rate
# 1/tau = A omega^4 + B omega^2 T exp(-C/T) for every branch.
SILICON_LIKE = {
    "kind": "quadratic",
    "T_eq": 300.0,
    "branches": [
        {"c1": 9.01e3, "c2": -2.0e-7, "degeneracy": 1.0},   # LA
        {"c1": 5.23e3, "c2": -2.26e-7, "degeneracy": 2.0},  # 2 x TA
    ],
    "a_lattice": 5.43e-10,
    "n_bins": 1000,
    "A": 1.32e-45,
    "B": 1.73e-19,
    "C": 137.0,
}

GRAY_UNIT = {"kind": "gray", "T_eq": 300.0, "v": 1.0, "tau": 1.0, "C": 1.0}


def _run(**kw):
    run = {
        "n_particles": 100_000,
        "seed": 0x5EED_1206_3316,
        "instance_id": 0,
        "max_scatter": 0,
        "max_events": 1 << 20,
        "n_bins_x": 0,
        "n_batch": 32,
        "t_final": 0.0,
        "sample_dt": 0.0,
        "grid": (0, 0, 0),
        "n_samples": 0,
        "n_hj": 0,
        "precision": "fp64",
    }
    run.update(kw)
    return run


def gray_slab(n_particles=100_000, kn=1.0, n_bins=50, seed=0x5EED_0000_0001,
              precision="fp64", walls=("black", "black"), dT=(1.0, -1.0), tau=None):
    """Gray 1D slab between isothermal black walls at T_eq +/- 1 K.

    Non-dimensional: v = C = 1, thickness L = 1, tau = Kn (so Lambda / L = Kn).
    Temperature and heat-flux profiles on ``n_bins`` bins.
    """
    mat = dict(GRAY_UNIT)
    mat["tau"] = float(kn if tau is None else tau)
    return {
        "material": mat,
        "geometry": {"kind": "planes", "L": 1.0, "wall_lo": walls[0], "wall_hi": walls[1]},
        "source": {"kind": "walls", "dT_lo": float(dT[0]), "dT_hi": float(dT[1])},
        "run": _run(n_particles=n_particles, seed=seed, n_bins_x=n_bins, precision=precision),
    }


def silicon_film(n_particles=10_000_000, thickness=100e-9, seed=0x5EED_0000_0002,
                 precision="fp32", max_scatter=40, max_events=4096, dTdz=-1.0e6,
                 material=None, walls=("diffuse", "diffuse"), n_hj=0, specularity=None):
    """Thin film with diffuse walls at x = 0 and x = thickness, driven by a
    uniform temperature gradient along z (in plane): in-plane conductivity.
    ``specularity`` = p makes both walls partially specular (specular with
    probability p, diffuse otherwise)."""
    geo = {"kind": "planes", "L": float(thickness), "wall_lo": walls[0], "wall_hi": walls[1]}
    if specularity is not None:
        geo.update(wall_lo="partial", wall_hi="partial", spec_lo=float(specularity), spec_hi=float(specularity))
    return {
        "material": copy.deepcopy(material or SILICON_LIKE),
        "geometry": geo,
        "source": {"kind": "gradient", "dTdz": float(dTdz)},
        "run": _run(n_particles=n_particles, seed=seed, max_scatter=max_scatter,
                    max_events=max_events, precision=precision, n_hj=n_hj),
    }


def bulk(n_particles=1_000_000, seed=0x5EED_0000_0003, precision="fp64", max_scatter=40,
         max_events=4096, material=None, dTdz=-1.0e6):
    """Infinite medium (no boundaries) under a uniform gradient along z."""
    return {
        "material": copy.deepcopy(material or SILICON_LIKE),
        "geometry": {"kind": "bulk"},
        "source": {"kind": "gradient", "dTdz": float(dTdz)},
        "run": _run(n_particles=n_particles, seed=seed, max_scatter=max_scatter,
                    max_events=max_events, precision=precision),
    }


def porous_film(n_particles=100_000_000, seed=0x5EED_0000_0004, precision="fp32",
                thickness=300e-9, pitch=100e-9, radius=30e-9, max_scatter=40,
                max_events=4096, material=None, n_hj=0, map=None, n_batch=16):
    """Periodic porous film: film normal x (thickness 300 nm, diffuse faces),
    cylindrical pores along x on a square lattice in (y, z) (pitch 100 nm,
    radius 30 nm, diffuse), 1 K across one period along z.  ``map=(ny, nz)``
    also asks for steady maps of T - T_eq(z) and the z flux over the unit cell
    (error bars from ``n_batch`` groups)."""
    run = _run(n_particles=n_particles, seed=seed, max_scatter=max_scatter,
               max_events=max_events, precision=precision, n_hj=n_hj)
    if map:
        run["map"] = (int(map[0]), int(map[1]))
        run["n_batch"] = int(n_batch)
    return {
        "material": copy.deepcopy(material or SILICON_LIKE),
        "geometry": {"kind": "porous", "L": float(thickness), "wall_lo": "diffuse",
                     "wall_hi": "diffuse", "pitch": float(pitch), "radius": float(radius),
                     "pore_wall": "diffuse", "cells_y": 1, "cells_z": 1},
        "source": {"kind": "gradient", "dTdz": -1.0 / float(pitch)},
        "run": run,
    }


def porous_pulse(n_particles=100_000_000, seed=0x5EED_0000_0005, precision="fp32",
                 grid=(32, 64, 64), n_samples=200, sample_dt=10e-12, t_final=2e-9,
                 cells=(6, 6), material=None, thickness=300e-9, pitch=100e-9, radius=30e-9,
                 max_events=1 << 20):
    """Transient: Gaussian surface heat pulse (lateral sigma 50 nm, duration
    sigma 100 ps centred at 300 ps) on the top face x = thickness of a 6 x 6
    cell periodic porous film; particle counts on a grid (nx along the
    thickness, ny x nz laterally) at ``n_samples`` times (k + 1/2) sample_dt."""
    Dy, Dz = pitch * cells[0], pitch * cells[1]
    return {
        "material": copy.deepcopy(material or SILICON_LIKE),
        "geometry": {"kind": "porous", "L": float(thickness), "wall_lo": "diffuse",
                     "wall_hi": "diffuse", "pitch": float(pitch), "radius": float(radius),
                     "pore_wall": "diffuse", "cells_y": int(cells[0]), "cells_z": int(cells[1])},
        "source": {"kind": "pulse", "sigma_x": 50e-9, "sigma_t": 100e-12, "t_center": 300e-12,
                   "energy": 1.0e-15, "y0": 0.5 * Dy - 0.5 * pitch, "z0": 0.5 * Dz - 0.5 * pitch},
        "run": _run(n_particles=n_particles, seed=seed, max_scatter=0, max_events=max_events,
                    precision=precision, t_final=float(t_final), sample_dt=float(sample_dt),
                    grid=tuple(int(g) for g in grid), n_samples=int(n_samples)),
    }


def porous_initial(n_particles=1_000_000, seed=0x5EED_0000_0007, precision="fp32", dT=1.0,
                   x_range=None, grid=(16, 8, 8), n_samples=50, sample_dt=20e-12, t_final=1e-9,
                   cells=(1, 1), material=None, thickness=300e-9, pitch=100e-9, radius=30e-9,
                   max_events=1 << 20):
    """Transient relaxation of an initial temperature excess dT in the layer
    x_range (default: the whole thickness) of a periodic porous film with
    adiabatic diffuse walls; particle counts on a grid at n_samples times."""
    lo, hi = x_range if x_range is not None else (0.0, thickness)
    return {
        "material": copy.deepcopy(material or SILICON_LIKE),
        "geometry": {"kind": "porous", "L": float(thickness), "wall_lo": "diffuse",
                     "wall_hi": "diffuse", "pitch": float(pitch), "radius": float(radius),
                     "pore_wall": "diffuse", "cells_y": int(cells[0]), "cells_z": int(cells[1])},
        "source": {"kind": "initial", "dT": float(dT), "x_lo": float(lo), "x_hi": float(hi)},
        "run": _run(n_particles=n_particles, seed=seed, max_scatter=0, max_events=max_events,
                    precision=precision, t_final=float(t_final), sample_dt=float(sample_dt),
                    grid=tuple(int(g) for g in grid), n_samples=int(n_samples)),
    }


def ttr_film(n_particles=2_000_000, seed=0x5EED_0000_0008, precision="fp32", dT=1.0, thickness=300e-9,
             heated=30e-9, nx=30, n_samples=100, sample_dt=50e-12, material=None, max_events=1 << 20):
    """Thermoreflectance-like transient on a single material: a film with
    adiabatic diffuse faces whose top layer (the last ``heated`` metres below
    x = thickness) starts dT above T_eq; the temperature of every x slab of
    the film is sampled at (k + 1/2) sample_dt.  (The paper's Al-on-Si
    experiment needs material data that is not available; one synthetic
    material stands in.)  A porous geometry with no pores is a film."""
    return porous_initial(n_particles=n_particles, seed=seed, precision=precision, dT=dT,
                          x_range=(thickness - heated, thickness), grid=(nx, 1, 1), n_samples=n_samples,
                          sample_dt=sample_dt, t_final=(n_samples + 1) * sample_dt, cells=(1, 1),
                          material=material, thickness=thickness, radius=0.0, max_events=max_events)


def batched_films(n_instances=256, seed=2012, n_min=1e4, n_max=1e7, L_min=10e-9, L_max=100e-6,
                  precision="fp32"):
    """Many silicon-like films of uneven size: thickness log-uniform in
    [10 nm, 100 um], particle counts log-uniform in [1e4, 1e7]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ls = np.exp(rng.uniform(math.log(L_min), math.log(L_max), n_instances))
    Ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_instances)).astype(np.int64)
    out = []
    for i in range(n_instances):
        p = silicon_film(n_particles=int(Ns[i]), thickness=float(Ls[i]),
                         seed=0x5EED_0000_0006, precision=precision)
        p["run"]["instance_id"] = i
        out.append(p)
    return out


def served_stream(duration_s=60.0, rate_hz=50.0, seed=2012, n_min=1e5, n_max=1e8,
                  targets=(0.01, 0.003)):
    """Poisson request stream mixing slab, film and porous-film problems with
    random sizes, T_eq in [100, 400] K and target relative standard errors
    (FP32 trajectories with FP64 tallies, as the request server traces them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        kind = int(rng.integers(0, 3))
        T_eq = float(rng.uniform(100.0, 400.0))
        budget = int(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        target = float(targets[int(rng.integers(0, len(targets)))])
        if kind == 0:
            kn = float(math.exp(rng.uniform(math.log(0.1), math.log(10.0))))
            p = gray_slab(n_particles=budget, kn=kn, n_bins=0, precision="fp32")
            p["material"]["T_eq"] = T_eq
        elif kind == 1:
            L = float(math.exp(rng.uniform(math.log(10e-9), math.log(100e-6))))
            p = silicon_film(n_particles=budget, thickness=L)
            p["material"]["T_eq"] = T_eq
        else:
            pitch = float(rng.uniform(50e-9, 200e-9))
            ratio = float(rng.uniform(0.1, 0.4))
            p = porous_film(n_particles=budget, pitch=pitch, radius=ratio * pitch)
            p["material"]["T_eq"] = T_eq
        p["run"]["instance_id"] = len(reqs)
        reqs.append({"arrival_s": t, "problem": p, "target_rel_err": target})
    return reqs


def with_run(problem, **kw):
    """Copy of ``problem`` with run parameters replaced."""
    p = copy.deepcopy(problem)
    p["run"].update(kw)
    return p
