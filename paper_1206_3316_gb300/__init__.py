"""GB300 (sm_103a) trajectory tracer for the linearized energy-based
deviational Monte Carlo method (Peraud & Hadjiconstantinou, arXiv:1206.3316).

The compute path is the CUDA library ``libLeMC.so`` (C ABI in
``include/le_mc.h``); this package only marshals arguments.  ``simulate`` runs
one problem described by a workload dict (see the ``workloads`` module):
material, geometry, source and run parameters.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    ARRAY, LeMcError, PARTICLE_DTYPE, geometry_desc, le_mc_abi_version, le_mc_alias_table,
    le_mc_create_geometry, le_mc_create_material, le_mc_destroy_geometry, le_mc_destroy_material,
    le_mc_destroy_run, le_mc_device_info, le_mc_last_error, le_mc_material_table, le_mc_philox,
    le_mc_read_array, le_mc_read_tallies, le_mc_run, le_mc_sample_modes, le_mc_wait, lib, material_desc,
    run_desc, LIB_PATH,
)


def simulate(problem, stream=None, arrays=True, record_particles=False, launch=None):
    """Create the material and geometry, run, read the tallies, destroy.

    Returns a dict with the scalar tallies (flux, kappa, psi, ... and the
    counters) and, when ``arrays``, the profile / H_j / grid arrays the problem
    asks for; per-particle records when ``record_particles``."""
    run = dict(problem["run"])
    if record_particles:
        run["record_particles"] = True
    mat = le_mc_create_material(material_desc(problem["material"]))
    try:
        geo = le_mc_create_geometry(geometry_desc(problem["geometry"]))
        try:
            h = le_mc_run(mat, geo, run_desc(problem["source"], run, launch), stream)
            try:
                out = le_mc_read_tallies(h)
                if arrays:
                    if run.get("n_bins_x", 0) > 0:
                        for k in ("T", "T_se", "q", "q_se"):
                            out[k] = le_mc_read_array(h, k)
                    if run.get("n_hj", 0) > 0:
                        out["H"] = le_mc_read_array(h, "H")
                        out["H_se"] = le_mc_read_array(h, "H_se")
                    if run.get("n_samples", 0) > 0:
                        gx, gy, gz = run["grid"]
                        out["grid"] = le_mc_read_array(h, "grid").reshape(run["n_samples"], gz, gy, gx)
                if record_particles:
                    out["particles_rec"] = le_mc_read_array(h, "particles")
                return out
            finally:
                le_mc_destroy_run(h)
        finally:
            le_mc_destroy_geometry(geo)
    finally:
        le_mc_destroy_material(mat)
