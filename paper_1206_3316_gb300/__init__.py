"""GB300 (sm_103a) trajectory tracer for the linearized energy-based
deviational Monte Carlo method (Peraud & Hadjiconstantinou, arXiv:1206.3316).

The compute path is the CUDA library ``libLeMC.so`` (C ABI in
``include/le_mc.h``); this package only marshals arguments.  ``simulate`` runs
one problem described by a workload dict (see the ``workloads`` module):
material, geometry, source and run parameters.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    ARRAY, LeMcError, PARTICLE_DTYPE, config_dict, geometry_desc, launch_config, le_mc_abi_version,
    le_mc_alias_table, le_mc_batch_autotune, le_mc_batch_create, le_mc_batch_destroy, le_mc_batch_launch,
    le_mc_batch_read, le_mc_batch_set_config, le_mc_batch_wait, le_mc_create_geometry, le_mc_create_material,
    le_mc_destroy_geometry, le_mc_destroy_material, le_mc_destroy_run, le_mc_device_info, le_mc_last_error,
    le_mc_material_table, le_mc_philox, le_mc_read_array, le_mc_read_tallies, le_mc_run, le_mc_sample_modes,
    le_mc_wait, lib, material_desc, run_desc, LIB_PATH, le_mc_server_cancel, le_mc_server_create,
    le_mc_server_destroy, le_mc_server_poll, le_mc_server_stats, le_mc_server_submit, le_mc_server_wait_all,
    le_mc_run_noalloc, le_mc_noalloc_flags, le_mc_truncation_study, le_mc_truncation_tail, NOALLOC_MAX_PARTICLES, le_mc_map_solid, le_mc_test_fail_allocation, DEVICE_FLAGS,
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
                        out["T_x"] = le_mc_read_array(h, "grid_Tx").reshape(run["n_samples"], gx)
                        out["T_x_se"] = le_mc_read_array(h, "grid_Tx_se").reshape(run["n_samples"], gx)
                    if tuple(run.get("map", (0, 0))) != (0, 0):
                        my, mz = run["map"]
                        for k in ("map_T", "map_T_se", "map_q", "map_q_se", "map_solid", "map_T_local"):
                            out[k] = le_mc_read_array(h, k).reshape(mz, my)
                if record_particles:
                    out["particles_rec"] = le_mc_read_array(h, "particles")
                return out
            finally:
                le_mc_destroy_run(h)
        finally:
            le_mc_destroy_geometry(geo)
    finally:
        le_mc_destroy_material(mat)


class Batch:
    """Many film or slab instances sharing one material, traced by one launch.

    ``problems`` are workload dicts that differ only in thickness, drive,
    particle count and instance id (see ``le_mc_batch_create``)."""

    def __init__(self, problems, config=None):
        if any(p["material"] != problems[0]["material"] for p in problems):
            raise ValueError("all instances of a batch share one material")
        self.problems = problems
        self.mat = le_mc_create_material(material_desc(problems[0]["material"]))
        try:
            self.h = le_mc_batch_create(self.mat, [geometry_desc(p["geometry"]) for p in problems],
                                        [run_desc(p["source"], p["run"]) for p in problems])
        except Exception:
            le_mc_destroy_material(self.mat)
            raise
        if config:
            le_mc_batch_set_config(self.h, config)

    def launch(self, stream=None):
        le_mc_batch_launch(self.h, stream)

    def wait(self):
        le_mc_batch_wait(self.h)

    def results(self):
        return [le_mc_batch_read(self.h, i) for i in range(len(self.problems))]

    def autotune(self, stream=None, cache_path=None):
        return le_mc_batch_autotune(self.h, stream, cache_path)

    def set_config(self, config):
        le_mc_batch_set_config(self.h, config)

    def close(self):
        if getattr(self, "h", None) is not None:
            le_mc_batch_destroy(self.h)
            self.h = None
        if getattr(self, "mat", None) is not None:
            le_mc_destroy_material(self.mat)
            self.mat = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request server (native worker thread).

    ``submit(problem, target_rel_err)`` queues a workload dict whose
    ``n_particles`` is the particle budget; ``poll`` returns its state and,
    once done, its normalised tallies over every particle traced."""

    def __init__(self, max_slots=8, hbm_budget_bytes=0, pilot_particles=0, max_epoch_particles=0, idle_exit_ms=0):
        self.h = le_mc_server_create(max_slots, hbm_budget_bytes, pilot_particles, max_epoch_particles, idle_exit_ms)

    def submit(self, problem, target_rel_err):
        return le_mc_server_submit(self.h, material_desc(problem["material"]), geometry_desc(problem["geometry"]),
                                   run_desc(problem["source"], problem["run"]), target_rel_err)

    def poll(self, rid):
        return le_mc_server_poll(self.h, rid)

    def cancel(self, rid):
        le_mc_server_cancel(self.h, rid)

    def wait_all(self, timeout_s=600.0):
        le_mc_server_wait_all(self.h, timeout_s)

    def stats(self):
        return le_mc_server_stats(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            le_mc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def truncation_study(H, H_se, resolved=3.0, first=2):
    """Choose the scattering cap K_s from the flux split by scattering index
    (the ``H`` / ``H_se`` arrays of a run with ``n_hj`` > 0), as the paper does
    empirically after its Fig. 2: <H_j> is the flux carried between the j-th
    and (j+1)-th relaxation of a history (j = 0: emission to the first).
    The arithmetic is the library's (le_mc_truncation_study); this wrapper
    returns a dict with
      k_s      the first j at which |<H_j>| falls to its own standard error;
      ratio    the geometric decay ratio of |<H_j>| fitted over the resolved,
               contiguous run of indices from ``first`` on (None if no fit);
      tail(K)  the flux the cap K drops, extrapolated from that fit."""
    import math

    t = le_mc_truncation_study(H, H_se, resolved, first)
    ratio = None if math.isnan(t.ratio) else float(t.ratio)
    return {"k_s": int(t.k_s), "ratio": ratio, "n_fit": int(t.n_fit),
            "tail": lambda K: le_mc_truncation_tail(t, K)}
