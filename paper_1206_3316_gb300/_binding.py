"""ctypes binding of the le_mc C ABI (``include/le_mc.h``).

Argument marshalling only: every step of the trajectory tracing runs in the
CUDA library.  Functions keep the C names; a non-OK status raises
``LeMcError`` carrying the status and ``le_mc_last_error()``.  The library is
loaded from the package directory; if it is missing, importing this module
fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LE_MC_LIBRARY selects another build of the library (the checking variant
# libLeMC_debug.so of build.build(debug=True)); there is no other backend
LIB_PATH = os.environ.get("LE_MC_LIBRARY") or os.path.join(_PKG, "libLeMC.so")

LE_MC_OK, LE_MC_ERR_INVALID, LE_MC_ERR_NOMEM, LE_MC_ERR_CUDA = 0, 1, 2, 3
LE_MC_ERR_TIMEOUT, LE_MC_ERR_BUDGET, LE_MC_ERR_STATE, LE_MC_ERR_NODEV = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "TIMEOUT", 5: "BUDGET", 6: "STATE", 7: "NODEV"}

MAT = {"gray": 0, "quadratic": 1, "tabulated": 2}
GEOM = {"planes": 0, "bulk": 1, "porous": 2}
WALL = {"black": 0, "diffuse": 1, "specular": 2, "partial": 3}
SRC = {"walls": 0, "gradient": 1, "pulse": 2, "initial": 3}
PREC = {"fp64": 0, "fp32": 1}
ARRAY = {"T": 0, "T_se": 1, "q": 2, "q_se": 3, "H": 4, "H_se": 5, "grid": 6, "particles": 7,
         "grid_T": 8, "grid_Tx": 9, "grid_T_se": 10, "grid_Tx_se": 11,
         "map_T": 12, "map_T_se": 13, "map_q": 14, "map_q_se": 15, "map_solid": 16, "map_T_local": 17}
MAX_BRANCHES = 4


class LeMcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"le_mc status {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class MaterialDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_branch", C.c_int32), ("n_bins", C.c_int32), ("n_modes", C.c_int32),
                ("T_eq", C.c_double), ("gray_v", C.c_double), ("gray_tau", C.c_double), ("gray_C", C.c_double),
                ("c1", C.c_double * MAX_BRANCHES), ("c2", C.c_double * MAX_BRANCHES),
                ("degeneracy", C.c_double * MAX_BRANCHES),
                ("a_lattice", C.c_double), ("A", C.c_double), ("B", C.c_double), ("C_exp", C.c_double),
                ("tab_v", C.POINTER(C.c_double)), ("tab_tau", C.POINTER(C.c_double)),
                ("tab_C", C.POINTER(C.c_double)), ("scatter_g", C.c_double)]


class GeometryDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("wall_lo", C.c_int32), ("wall_hi", C.c_int32), ("pore_wall", C.c_int32),
                ("L", C.c_double), ("pitch", C.c_double), ("radius", C.c_double),
                ("cells_y", C.c_int32), ("cells_z", C.c_int32),
                ("spec_lo", C.c_double), ("spec_hi", C.c_double), ("spec_pore", C.c_double)]


class RunDesc(C.Structure):
    _fields_ = [("source", C.c_int32), ("precision", C.c_int32),
                ("dT_lo", C.c_double), ("dT_hi", C.c_double), ("dTdz", C.c_double),
                ("pulse_sigma_x", C.c_double), ("pulse_sigma_t", C.c_double), ("pulse_t_center", C.c_double),
                ("pulse_energy", C.c_double), ("pulse_y0", C.c_double), ("pulse_z0", C.c_double),
                ("n_particles", C.c_uint64), ("seed", C.c_uint64),
                ("instance_id", C.c_uint32), ("max_scatter", C.c_uint32), ("max_events", C.c_uint32),
                ("n_bins_x", C.c_int32), ("n_batch", C.c_int32),
                ("grid_nx", C.c_int32), ("grid_ny", C.c_int32), ("grid_nz", C.c_int32), ("n_samples", C.c_int32),
                ("t_final", C.c_double), ("sample_dt", C.c_double),
                ("n_hj", C.c_int32), ("record_particles", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("threads_per_block", C.c_int32),
                ("schedule", C.c_int32), ("refill_min", C.c_int32), ("long_mfp_cut", C.c_double),
                ("chunk", C.c_int32), ("first_particle", C.c_uint32),
                ("init_dT", C.c_double), ("init_x_lo", C.c_double), ("init_x_hi", C.c_double),
                ("max_collisions", C.c_uint32), ("map_ny", C.c_int32), ("map_nz", C.c_int32)]


class Tallies(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "P_total", "E_eff_dot", "E_eff", "C_tot", "sum_sL", "sum_sL2", "flux", "flux_se", "kappa",
        "kappa_se", "kappa_solid", "psi", "psi_se")] + [
        (n, C.c_uint64) for n in ("particles", "segments", "scatters", "wall_hits", "periodic",
                                  "truncated", "absorbed")] + [
        ("kernel_ms", C.c_double), ("prepass_ms", C.c_double), ("kernel_launches", C.c_uint32),
        ("device_flags", C.c_uint32), ("long_listed", C.c_uint32), ("extreme_traced", C.c_uint32)]


class Particle(C.Structure):
    _fields_ = [("sign", C.c_int8), ("fate", C.c_int8), ("pad", C.c_int16),
                ("n_seg", C.c_uint32), ("n_scat", C.c_uint32), ("n_wall", C.c_uint32),
                ("n_periodic", C.c_uint32), ("mode0", C.c_uint32),
                ("L_axis", C.c_double), ("x0", C.c_double), ("t0", C.c_double)]


class LaunchConfig(C.Structure):
    _fields_ = [("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("refill_min", C.c_int32),
                ("chunk", C.c_int32), ("use_graph", C.c_int32), ("ms", C.c_float)]


class ServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("pad", C.c_int32), ("hbm_budget_bytes", C.c_uint64),
                ("pilot_particles", C.c_uint64), ("max_epoch_particles", C.c_uint64), ("idle_exit_ms", C.c_int32),
                ("pad2", C.c_int32)]


class RequestStatus(C.Structure):
    _fields_ = [("state", C.c_int32), ("epochs", C.c_int32), ("submit_s", C.c_double), ("start_s", C.c_double),
                ("done_s", C.c_double), ("rel_err", C.c_double), ("tallies", Tallies)]


class ServerCounters(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "failed", "active", "queued", "segments",
                                          "particles", "hbm_in_use")] + [("uptime_s", C.c_double),
                                                                         ("kernel_launches", C.c_uint64)]


REQUEST_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}

PARTICLE_DTYPE = np.dtype([("sign", np.int8), ("fate", np.int8), ("pad", np.int16),
                           ("n_seg", np.uint32), ("n_scat", np.uint32), ("n_wall", np.uint32),
                           ("n_periodic", np.uint32), ("mode0", np.uint32),
                           ("L_axis", np.float64), ("x0", np.float64), ("t0", np.float64)])

_STATUS = C.c_int
_H = C.c_void_p

# name -> (restype, argtypes)
class Truncation(C.Structure):
    _fields_ = [("k_s", C.c_int32), ("n_fit", C.c_int32), ("ratio", C.c_double), ("amp", C.c_double),
                ("sign", C.c_double)]


SIGNATURES = {
    "le_mc_create_material": (_STATUS, [C.POINTER(MaterialDesc), C.POINTER(_H)]),
    "le_mc_destroy_material": (_STATUS, [_H]),
    "le_mc_material_table": (_STATUS, [C.POINTER(MaterialDesc), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "le_mc_alias_table": (_STATUS, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "le_mc_map_solid": (_STATUS, [C.POINTER(GeometryDesc), C.c_int32, C.c_int32, C.c_void_p]),
    "le_mc_test_fail_allocation": (_STATUS, [C.c_int32]),
    "le_mc_create_geometry": (_STATUS, [C.POINTER(GeometryDesc), C.POINTER(_H)]),
    "le_mc_destroy_geometry": (_STATUS, [_H]),
    "le_mc_run": (_STATUS, [_H, _H, C.POINTER(RunDesc), C.c_void_p, C.POINTER(_H)]),
    "le_mc_wait": (_STATUS, [_H]),
    "le_mc_read_tallies": (_STATUS, [_H, C.POINTER(Tallies)]),
    "le_mc_read_array": (_STATUS, [_H, C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "le_mc_destroy_run": (_STATUS, [_H]),
    "le_mc_philox": (_STATUS, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_size_t]),
    "le_mc_sample_modes": (_STATUS, [_H, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t]),
    "le_mc_device_info": (_STATUS, [C.POINTER(C.c_int32), C.c_char_p, C.c_size_t]),
    "le_mc_batch_create": (_STATUS, [_H, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(_H)]),
    "le_mc_batch_set_config": (_STATUS, [_H, C.POINTER(LaunchConfig)]),
    "le_mc_batch_launch": (_STATUS, [_H, C.c_void_p]),
    "le_mc_batch_wait": (_STATUS, [_H]),
    "le_mc_batch_read": (_STATUS, [_H, C.c_int32, C.POINTER(Tallies)]),
    "le_mc_batch_autotune": (_STATUS, [_H, C.c_void_p, C.c_char_p, C.POINTER(LaunchConfig)]),
    "le_mc_batch_destroy": (_STATUS, [_H]),
    "le_mc_server_create": (_STATUS, [C.POINTER(ServerConfig), C.POINTER(_H)]),
    "le_mc_server_submit": (_STATUS, [_H, C.POINTER(MaterialDesc), C.POINTER(GeometryDesc), C.POINTER(RunDesc),
                                      C.c_double, C.POINTER(C.c_uint64)]),
    "le_mc_server_poll": (_STATUS, [_H, C.c_uint64, C.POINTER(RequestStatus)]),
    "le_mc_server_cancel": (_STATUS, [_H, C.c_uint64]),
    "le_mc_server_wait_all": (_STATUS, [_H, C.c_double]),
    "le_mc_server_stats": (_STATUS, [_H, C.POINTER(ServerCounters)]),
    "le_mc_server_destroy": (_STATUS, [_H]),
    "le_mc_run_noalloc": (_STATUS, [_H, _H, C.POINTER(RunDesc), C.c_void_p, C.c_void_p, C.c_void_p]),
    "le_mc_noalloc_flags": (_STATUS, [C.c_void_p, C.POINTER(C.c_uint32)]),
    "le_mc_truncation_study": (_STATUS, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_int32,
                                         C.POINTER(Truncation)]),
    "le_mc_truncation_tail": (_STATUS, [C.POINTER(Truncation), C.c_int32, C.POINTER(C.c_double)]),
    "le_mc_struct_size": (C.c_int32, [C.c_int32]),
    "le_mc_last_error": (C.c_char_p, []),
    "le_mc_abi_version": (C.c_int32, []),
}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"le_mc CUDA library not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python -m paper_1206_3316_gb300.build")
lib = C.CDLL(LIB_PATH)
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

for _i, _cls in enumerate((MaterialDesc, GeometryDesc, RunDesc, Tallies, Particle, LaunchConfig)):
    if lib.le_mc_struct_size(_i) != C.sizeof(_cls):
        raise ImportError(f"ABI mismatch: {_cls.__name__} is {C.sizeof(_cls)} bytes in Python, "
                          f"{lib.le_mc_struct_size(_i)} in libLeMC.so")


def _check(status, what):
    if status != LE_MC_OK:
        raise LeMcError(status, f"{what}: {lib.le_mc_last_error().decode(errors='replace')}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


# ---- descriptors from workload dicts -------------------------------------
def material_desc(mat):
    d = MaterialDesc()
    d.kind = MAT[mat["kind"]]
    d.T_eq = float(mat.get("T_eq", 300.0))
    d.scatter_g = float(mat.get("scatter_g", 0.0))
    keep = []
    if mat["kind"] == "gray":
        d.gray_v, d.gray_tau, d.gray_C = mat["v"], mat["tau"], mat["C"]
    elif mat["kind"] == "quadratic":
        br = mat["branches"]
        d.n_branch = len(br)
        for i, b in enumerate(br):
            d.c1[i], d.c2[i], d.degeneracy[i] = b["c1"], b["c2"], b["degeneracy"]
        d.n_bins = int(mat["n_bins"])
        d.a_lattice, d.A, d.B, d.C_exp = mat["a_lattice"], mat["A"], mat["B"], mat["C"]
    else:
        arrs = [np.ascontiguousarray(mat[k], dtype=np.float64) for k in ("v", "tau", "C")]
        keep = arrs
        d.n_modes = arrs[0].size
        d.tab_v, d.tab_tau, d.tab_C = (a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs)
    d._keep = keep
    return d


def geometry_desc(geo):
    g = GeometryDesc()
    g.kind = GEOM[geo["kind"]]
    g.wall_lo = WALL[geo.get("wall_lo", "diffuse")]
    g.wall_hi = WALL[geo.get("wall_hi", "diffuse")]
    g.pore_wall = WALL[geo.get("pore_wall", "diffuse")]
    g.L = float(geo.get("L", 0.0))
    g.pitch = float(geo.get("pitch", 0.0))
    g.radius = float(geo.get("radius", 0.0))
    g.cells_y = int(geo.get("cells_y", 1))
    g.cells_z = int(geo.get("cells_z", 1))
    g.spec_lo = float(geo.get("spec_lo", 0.0))
    g.spec_hi = float(geo.get("spec_hi", 0.0))
    g.spec_pore = float(geo.get("spec_pore", 0.0))
    return g


def run_desc(src, run, launch=None):
    r = RunDesc()
    r.source = SRC[src["kind"]]
    r.precision = PREC[run.get("precision", "fp64")]
    r.dT_lo, r.dT_hi, r.dTdz = src.get("dT_lo", 0.0), src.get("dT_hi", 0.0), src.get("dTdz", 0.0)
    r.pulse_sigma_x, r.pulse_sigma_t = src.get("sigma_x", 0.0), src.get("sigma_t", 0.0)
    r.pulse_t_center, r.pulse_energy = src.get("t_center", 0.0), src.get("energy", 0.0)
    r.pulse_y0, r.pulse_z0 = src.get("y0", 0.0), src.get("z0", 0.0)
    r.n_particles, r.seed = int(run["n_particles"]), int(run["seed"])
    r.instance_id = int(run.get("instance_id", 0))
    r.max_scatter, r.max_events = int(run.get("max_scatter", 0)), int(run.get("max_events", 1 << 20))
    r.n_bins_x, r.n_batch = int(run.get("n_bins_x", 0)), int(run.get("n_batch", 32))
    gx, gy, gz = run.get("grid", (0, 0, 0))
    r.grid_nx, r.grid_ny, r.grid_nz = int(gx), int(gy), int(gz)
    r.n_samples = int(run.get("n_samples", 0))
    r.t_final, r.sample_dt = float(run.get("t_final", 0.0)), float(run.get("sample_dt", 0.0))
    r.n_hj = int(run.get("n_hj", 0))
    r.record_particles = 1 if run.get("record_particles", False) else 0
    launch = launch or {}
    r.blocks_per_sm = int(launch.get("blocks_per_sm", run.get("blocks_per_sm", 0)))
    r.threads_per_block = int(launch.get("threads_per_block", run.get("threads_per_block", 0)))
    r.schedule = {"auto": 0, "long_first": 1, "natural": 2}[launch.get("schedule", run.get("schedule", "auto"))]
    r.long_mfp_cut = float(launch.get("long_mfp_cut", run.get("long_mfp_cut", 0.0)))
    r.refill_min = int(launch.get("refill_min", run.get("refill_min", 0)))
    r.chunk = int(launch.get("chunk", run.get("chunk", 0)))
    r.first_particle = int(run.get("first_particle", 0))
    r.max_collisions = int(run.get("max_collisions", 0))
    r.init_dT = float(src.get("dT", 0.0)) if src["kind"] == "initial" else 0.0
    r.init_x_lo, r.init_x_hi = float(src.get("x_lo", 0.0)), float(src.get("x_hi", 0.0))
    my, mz = run.get("map", (0, 0))
    r.map_ny, r.map_nz = int(my), int(mz)
    return r


# ---- thin wrappers with the C names --------------------------------------
def le_mc_create_material(desc):
    h = _H()
    _check(lib.le_mc_create_material(C.byref(desc), C.byref(h)), "le_mc_create_material")
    return h


def le_mc_destroy_material(h):
    _check(lib.le_mc_destroy_material(h), "le_mc_destroy_material")


def le_mc_material_table(desc):
    n = C.c_int32()
    _check(lib.le_mc_material_table(C.byref(desc), None, None, None, None, 0, C.byref(n)), "le_mc_material_table")
    arrs = [np.zeros(n.value) for _ in range(4)]
    _check(lib.le_mc_material_table(C.byref(desc), *[a.ctypes.data for a in arrs], n.value, C.byref(n)),
           "le_mc_material_table")
    return tuple(arrs)


def le_mc_alias_table(weights):
    w = np.ascontiguousarray(weights, dtype=np.float64)
    thr = np.zeros(w.size, dtype=np.uint32)
    al = np.zeros(w.size, dtype=np.uint32)
    _check(lib.le_mc_alias_table(w.ctypes.data, w.size, thr.ctypes.data, al.ctypes.data), "le_mc_alias_table")
    return thr, al


def le_mc_map_solid(desc, map_ny, map_nz):
    out = np.zeros((int(map_nz), int(map_ny)))
    _check(lib.le_mc_map_solid(C.byref(desc), int(map_ny), int(map_nz), out.ctypes.data), "le_mc_map_solid")
    return out


def le_mc_test_fail_allocation(after):
    _check(lib.le_mc_test_fail_allocation(int(after)), "le_mc_test_fail_allocation")


DEVICE_FLAGS = {"rejection_exhausted": 1, "bad_launch": 4}


def le_mc_create_geometry(desc):
    h = _H()
    _check(lib.le_mc_create_geometry(C.byref(desc), C.byref(h)), "le_mc_create_geometry")
    return h


def le_mc_destroy_geometry(h):
    _check(lib.le_mc_destroy_geometry(h), "le_mc_destroy_geometry")


def le_mc_run(mat, geo, desc, stream=None):
    h = _H()
    st = lib.le_mc_run(mat, geo, C.byref(desc), _stream_ptr(stream), C.byref(h))
    if st != LE_MC_OK:
        msg = lib.le_mc_last_error().decode(errors="replace")
        if h.value:
            lib.le_mc_destroy_run(h)
        raise LeMcError(st, f"le_mc_run: {msg}")
    return h


def le_mc_wait(h):
    _check(lib.le_mc_wait(h), "le_mc_wait")


def le_mc_read_tallies(h):
    t = Tallies()
    _check(lib.le_mc_read_tallies(h, C.byref(t)), "le_mc_read_tallies")
    return {f[0]: getattr(t, f[0]) for f in Tallies._fields_}


def le_mc_read_array(h, which):
    code = ARRAY[which]
    n = C.c_size_t()
    _check(lib.le_mc_read_array(h, code, None, 0, C.byref(n)), "le_mc_read_array")
    if which == "grid":
        out = np.zeros(n.value // 4, dtype=np.int32)
    elif which == "particles":
        out = np.zeros(n.value // PARTICLE_DTYPE.itemsize, dtype=PARTICLE_DTYPE)
    else:
        out = np.zeros(n.value // 8, dtype=np.float64)
    _check(lib.le_mc_read_array(h, code, out.ctypes.data, out.nbytes, C.byref(n)), "le_mc_read_array")
    return out


def le_mc_destroy_run(h):
    _check(lib.le_mc_destroy_run(h), "le_mc_destroy_run")


def le_mc_philox(counters, key0, key1):
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    _check(lib.le_mc_philox(c.ctypes.data, int(key0), int(key1), out.ctypes.data, c.shape[0]), "le_mc_philox")
    return out


def le_mc_sample_modes(mat, which, words):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros(w.size, dtype=np.int32)
    _check(lib.le_mc_sample_modes(mat, 1 if which in (1, "scatter") else 0, w.ctypes.data, out.ctypes.data, w.size),
           "le_mc_sample_modes")
    return out


def le_mc_device_info():
    n = C.c_int32()
    buf = C.create_string_buffer(256)
    _check(lib.le_mc_device_info(C.byref(n), buf, 256), "le_mc_device_info")
    return n.value, buf.value.decode()


def le_mc_last_error():
    return lib.le_mc_last_error().decode(errors="replace")


def le_mc_abi_version():
    return lib.le_mc_abi_version()


def launch_config(cfg=None):
    c = LaunchConfig()
    cfg = cfg or {}
    c.threads_per_block = int(cfg.get("threads_per_block", 0))
    c.blocks_per_sm = int(cfg.get("blocks_per_sm", 0))
    c.refill_min = int(cfg.get("refill_min", 0))
    c.chunk = int(cfg.get("chunk", 0))
    c.use_graph = 1 if cfg.get("use_graph", False) else 0
    return c


def config_dict(c):
    return {"threads_per_block": c.threads_per_block, "blocks_per_sm": c.blocks_per_sm,
            "refill_min": c.refill_min, "chunk": c.chunk, "use_graph": bool(c.use_graph), "ms": c.ms}


def le_mc_batch_create(mat, geoms, runs):
    n = len(geoms)
    g = (GeometryDesc * n)(*geoms)
    r = (RunDesc * n)(*runs)
    h = _H()
    _check(lib.le_mc_batch_create(mat, n, C.cast(g, C.c_void_p), C.cast(r, C.c_void_p), C.byref(h)),
           "le_mc_batch_create")
    return h


def le_mc_batch_set_config(b, cfg):
    _check(lib.le_mc_batch_set_config(b, C.byref(launch_config(cfg) if isinstance(cfg, dict) else cfg)),
           "le_mc_batch_set_config")


def le_mc_batch_launch(b, stream=None):
    _check(lib.le_mc_batch_launch(b, _stream_ptr(stream)), "le_mc_batch_launch")


def le_mc_batch_wait(b):
    _check(lib.le_mc_batch_wait(b), "le_mc_batch_wait")


def le_mc_batch_read(b, i):
    t = Tallies()
    _check(lib.le_mc_batch_read(b, i, C.byref(t)), "le_mc_batch_read")
    return {f[0]: getattr(t, f[0]) for f in Tallies._fields_}


def le_mc_batch_autotune(b, stream=None, cache_path=None):
    c = LaunchConfig()
    path = cache_path.encode() if cache_path else None
    _check(lib.le_mc_batch_autotune(b, _stream_ptr(stream), path, C.byref(c)), "le_mc_batch_autotune")
    return config_dict(c)


def le_mc_batch_destroy(b):
    _check(lib.le_mc_batch_destroy(b), "le_mc_batch_destroy")


def le_mc_server_create(max_slots=0, hbm_budget_bytes=0, pilot_particles=0, max_epoch_particles=0, idle_exit_ms=0):
    c = ServerConfig()
    c.max_slots, c.hbm_budget_bytes = int(max_slots), int(hbm_budget_bytes)
    c.pilot_particles, c.max_epoch_particles = int(pilot_particles), int(max_epoch_particles)
    c.idle_exit_ms = int(idle_exit_ms)
    h = _H()
    _check(lib.le_mc_server_create(C.byref(c), C.byref(h)), "le_mc_server_create")
    return h


def le_mc_server_submit(s, mdesc, gdesc, rdesc, target_rel_err):
    rid = C.c_uint64()
    _check(lib.le_mc_server_submit(s, C.byref(mdesc), C.byref(gdesc), C.byref(rdesc), float(target_rel_err),
                                   C.byref(rid)), "le_mc_server_submit")
    return rid.value


def le_mc_server_poll(s, rid):
    st = RequestStatus()
    _check(lib.le_mc_server_poll(s, int(rid), C.byref(st)), "le_mc_server_poll")
    out = {"state": REQUEST_STATES[st.state], "epochs": st.epochs, "submit_s": st.submit_s,
           "start_s": st.start_s, "done_s": st.done_s, "rel_err": st.rel_err}
    out.update({f[0]: getattr(st.tallies, f[0]) for f in Tallies._fields_})
    return out


def le_mc_server_cancel(s, rid):
    _check(lib.le_mc_server_cancel(s, int(rid)), "le_mc_server_cancel")


def le_mc_server_wait_all(s, timeout_s):
    _check(lib.le_mc_server_wait_all(s, float(timeout_s)), "le_mc_server_wait_all")


def le_mc_server_stats(s):
    c = ServerCounters()
    _check(lib.le_mc_server_stats(s, C.byref(c)), "le_mc_server_stats")
    return {f[0]: getattr(c, f[0]) for f in ServerCounters._fields_}


def le_mc_server_destroy(s):
    _check(lib.le_mc_server_destroy(s), "le_mc_server_destroy")


NOALLOC_MAX_PARTICLES = 1 << 22


def le_mc_run_noalloc(mat, geo, desc, d_sums, d_counters, stream=None):
    """Trace without allocating: d_sums (2 doubles) and d_counters (7 uint64)
    are device addresses owned by the caller (ints, e.g. tensor.data_ptr())."""
    _check(lib.le_mc_run_noalloc(mat, geo, C.byref(desc), int(d_sums), int(d_counters), _stream_ptr(stream)),
           "le_mc_run_noalloc")


def le_mc_noalloc_flags(stream=None):
    """Device status bits (LE_MC_FLAG_*) of the last le_mc_run_noalloc call on
    the current device, after `stream` has finished."""
    f = C.c_uint32(0)
    _check(lib.le_mc_noalloc_flags(_stream_ptr(stream), C.byref(f)), "le_mc_noalloc_flags")
    return int(f.value)


def le_mc_truncation_study(H, H_se, resolved=3.0, first=2):
    """Host-only study of the flux split by scattering index (see
    include/le_mc.h): returns the le_mc_truncation fields as a dict."""
    import numpy as np
    H = np.ascontiguousarray(H, dtype=np.float64)
    se = np.ascontiguousarray(H_se, dtype=np.float64)
    if H.shape != se.shape or H.ndim != 1:
        raise ValueError("H and H_se must be 1-D arrays of one length")
    t = Truncation()
    _check(lib.le_mc_truncation_study(H.ctypes.data, se.ctypes.data, int(H.size), float(resolved), int(first),
                                      C.byref(t)), "le_mc_truncation_study")
    return t


def le_mc_truncation_tail(study, K):
    d = C.c_double(0.0)
    _check(lib.le_mc_truncation_tail(C.byref(study), int(K), C.byref(d)), "le_mc_truncation_tail")
    return float(d.value)
