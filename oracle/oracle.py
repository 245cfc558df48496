"""ctypes wrapper around the FP64 CPU oracle (``le_mc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product package.

Pins (what each oracle function is checked against in the ``-m "not gpu"``
tests, none of which re-derives the oracle's own formulas):

* Philox4x32-10: NVIDIA's readable curand header function, compiled for the
  host, on fixed counters and keys (bit-exact).
* Inverse-CDF mode draws: exact bin probabilities (chi-square on 1e6 draws)
  and monotonicity.
* Emission: cosine-law moments E[mu] = 2/3, E[mu^2] = 1/2; |mu|-weighted
  gradient source moments; uniform positions; sign balance (Eq. 6).
* Gray slab (black walls): heat flux Psi and bin-averaged temperature against
  a deterministic product-integration solution of the integral equation of
  the slab (``analytic.py``), the ballistic limit Psi = 1, the per-particle
  invariant s L_x / L in {0, 1}, antisymmetry of T(x).
* Films with diffuse walls: conductivity against the Fuchs-Sondheimer sum
  (the analytic thin-film solution) and the bulk sum (1/3) sum C v^2 tau;
  vanishing mean contribution after the first event.
* Porous film: ray-cylinder intersections against brute-force marching,
  bounds and mirror symmetry; transient energy conservation (exact); its
  first-event and first-free-path conductivities against quasi-Monte Carlo
  means of each particle's closed-form first-flight contribution; the pore
  wall's Lambertian re-emission by the invariance of a uniform isotropic
  excess in a pored cell (counts stay in proportion to the solid volume and
  whole; a law uniform in the cosine, or about the wrong normal, fails it).
  The full (untruncated) porous-film conductivity has no closed form: parity
  unpinned.  What bounds it: the zero-radius limit (the Fuchs-Sondheimer
  film), the upper bound kappa_film (1 - porosity), the first-event and
  first-free-path pins above (same emission law, signs and normalisation),
  the pinned pore-wall law, and the flux split by scattering index, whose
  tail the truncation study extrapolates.
* Steady maps over the unit cell: solid fractions against the exact total
  and point counts; the flux map partitions the scalar flux; the unit
  cell's mirror symmetries; flat maps for a film without pores.
* Transient estimator: free streaming between specular faces (slab
  fractions from the unfolded kinematics); pulse emission times (truncated
  Gaussian law) and lateral law (Rayleigh radius, cosine directions).
* Film depth profile of the in-plane flux: the depth form of the thin-film
  solution.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "le_mc_oracle.c")
_LIB = os.path.join(_HERE, "liblemc_oracle.so")

MAT = {"gray": 0, "quadratic": 1}
GEOM = {"planes": 0, "bulk": 1, "porous": 2}
WALL = {"black": 0, "diffuse": 1, "specular": 2, "partial": 3}
SRC = {"walls": 0, "gradient": 1, "pulse": 2, "initial": 3}
FATE = {0: "absorbed", 1: "max_scatter", 2: "max_events", 3: "t_final", 4: "max_collisions"}


class Problem(C.Structure):
    _fields_ = [
        ("mat_kind", C.c_int32), ("n_branch", C.c_int32), ("n_bins_omega", C.c_int32), ("pad0", C.c_int32),
        ("T_eq", C.c_double), ("gray_v", C.c_double), ("gray_tau", C.c_double), ("gray_C", C.c_double),
        ("c1", C.c_double * 4), ("c2", C.c_double * 4), ("degeneracy", C.c_double * 4),
        ("a_lattice", C.c_double), ("A", C.c_double), ("B", C.c_double), ("Cexp", C.c_double),
        ("scatter_g", C.c_double),
        ("geom_kind", C.c_int32), ("wall_lo", C.c_int32), ("wall_hi", C.c_int32), ("pore_wall", C.c_int32),
        ("L", C.c_double), ("pitch", C.c_double), ("radius", C.c_double),
        ("cells_y", C.c_int32), ("cells_z", C.c_int32),
        ("spec_lo", C.c_double), ("spec_hi", C.c_double), ("spec_pore", C.c_double),
        ("src_kind", C.c_int32), ("pad1", C.c_int32),
        ("dT_lo", C.c_double), ("dT_hi", C.c_double), ("dTdz", C.c_double),
        ("pulse_sigma_x", C.c_double), ("pulse_sigma_t", C.c_double), ("pulse_t_center", C.c_double),
        ("pulse_energy", C.c_double), ("pulse_y0", C.c_double), ("pulse_z0", C.c_double),
        ("init_dT", C.c_double), ("init_x_lo", C.c_double), ("init_x_hi", C.c_double),
        ("n_particles", C.c_uint64), ("seed", C.c_uint64),
        ("instance_id", C.c_uint32), ("max_scatter", C.c_uint32), ("max_events", C.c_uint32),
        ("max_collisions", C.c_uint32),
        ("n_bins_x", C.c_int32), ("n_batch", C.c_int32),
        ("grid_nx", C.c_int32), ("grid_ny", C.c_int32), ("grid_nz", C.c_int32), ("n_samples", C.c_int32),
        ("n_hj", C.c_int32),
        ("t_final", C.c_double), ("sample_dt", C.c_double),
        ("n_threads", C.c_int32), ("record_particles", C.c_int32),
        ("map_ny", C.c_int32), ("map_nz", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "P_total", "E_eff_dot", "E_eff", "C_tot", "sum_sL", "sum_sL2", "flux", "flux_se",
        "kappa", "kappa_se", "kappa_solid", "psi", "psi_se")] + [
        (n, C.c_uint64) for n in ("particles", "segments", "scatters", "wall_hits", "periodic",
                                  "truncated", "absorbed")]


class Particle(C.Structure):
    _fields_ = [("sign", C.c_int8), ("fate", C.c_int8), ("pad", C.c_int16),
                ("n_seg", C.c_uint32), ("n_scat", C.c_uint32), ("n_wall", C.c_uint32),
                ("n_periodic", C.c_uint32), ("mode0", C.c_uint32),
                ("L_axis", C.c_double), ("x0", C.c_double), ("t0", C.c_double)]


PARTICLE_DTYPE = np.dtype([("sign", np.int8), ("fate", np.int8), ("pad", np.int16),
                           ("n_seg", np.uint32), ("n_scat", np.uint32), ("n_wall", np.uint32),
                           ("n_periodic", np.uint32), ("mode0", np.uint32),
                           ("L_axis", np.float64), ("x0", np.float64), ("t0", np.float64)])


def build(force=False):
    """Compile the oracle with the host C compiler (no CUDA involved).

    ``-ffp-contract=off`` keeps every product and sum separately rounded, so
    the oracle gives the same bits on x86-64 and aarch64 hosts."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _bind(handle):
    handle.orc_run.restype = C.c_int
    handle.orc_run.argtypes = [C.POINTER(Problem), C.POINTER(Result)] + [C.c_void_p] * 9
    handle.orc_emit.restype = C.c_int
    handle.orc_emit.argtypes = [C.POINTER(Problem), C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]
    return handle


def load_variant(path):
    """A separately compiled copy of the oracle (used by the tests that plant
    mistakes in a copy of the source to show that the pins catch them)."""
    return _bind(C.CDLL(path))


def compile_variant(source_text, out_path):
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", out_path, src, "-lm", "-lpthread"], check=True)
    return load_variant(out_path)


def source_text():
    with open(_SRC) as fh:
        return fh.read()


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_run.restype = C.c_int
        _lib.orc_run.argtypes = [C.POINTER(Problem), C.POINTER(Result)] + [C.c_void_p] * 9
        _lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        _lib.orc_material.restype = C.c_int
        _lib.orc_material.argtypes = [C.POINTER(Problem)] + [C.c_void_p] * 4 + [C.c_int]
        _lib.orc_draw_modes.restype = C.c_int
        _lib.orc_draw_modes.argtypes = [C.POINTER(Problem), C.c_int, C.c_void_p, C.c_int, C.c_void_p]
        _lib.orc_first_boundary.restype = C.c_double
        _lib.orc_first_boundary.argtypes = [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]
        _lib.orc_scatter_direction.restype = None
        _lib.orc_scatter_direction.argtypes = [C.c_double, C.c_void_p, C.c_double, C.c_double, C.c_void_p]
        _lib.orc_emit.restype = C.c_int
        _lib.orc_emit.argtypes = [C.POINTER(Problem), C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]
        assert _lib.orc_sizeof_problem() == C.sizeof(Problem)
        assert _lib.orc_sizeof_result() == C.sizeof(Result)
        assert _lib.orc_sizeof_particle() == C.sizeof(Particle) == PARTICLE_DTYPE.itemsize
    return _lib


def to_problem(prob, n_threads=None, record_particles=False):
    """Flatten a workload dict (see ``workloads``) into the oracle's struct."""
    m, g, s, r = prob["material"], prob["geometry"], prob["source"], prob["run"]
    p = Problem()
    p.mat_kind = MAT[m["kind"]]
    p.T_eq = m.get("T_eq", 300.0)
    if m["kind"] == "gray":
        p.gray_v, p.gray_tau, p.gray_C = m["v"], m["tau"], m["C"]
    else:
        br = m["branches"]
        p.n_branch = len(br)
        for i, b in enumerate(br):
            p.c1[i], p.c2[i], p.degeneracy[i] = b["c1"], b["c2"], b["degeneracy"]
        p.n_bins_omega = m["n_bins"]
        p.a_lattice, p.A, p.B, p.Cexp = m["a_lattice"], m["A"], m["B"], m["C"]
    p.scatter_g = m.get("scatter_g", 0.0)
    p.geom_kind = GEOM[g["kind"]]
    p.L = g.get("L", 0.0)
    p.wall_lo = WALL[g.get("wall_lo", "diffuse")]
    p.wall_hi = WALL[g.get("wall_hi", "diffuse")]
    p.pore_wall = WALL[g.get("pore_wall", "diffuse")]
    p.pitch, p.radius = g.get("pitch", 0.0), g.get("radius", 0.0)
    p.cells_y, p.cells_z = g.get("cells_y", 1), g.get("cells_z", 1)
    p.spec_lo, p.spec_hi, p.spec_pore = g.get("spec_lo", 0.0), g.get("spec_hi", 0.0), g.get("spec_pore", 0.0)
    p.src_kind = SRC[s["kind"]]
    p.dT_lo, p.dT_hi, p.dTdz = s.get("dT_lo", 0.0), s.get("dT_hi", 0.0), s.get("dTdz", 0.0)
    p.pulse_sigma_x, p.pulse_sigma_t = s.get("sigma_x", 0.0), s.get("sigma_t", 0.0)
    p.pulse_t_center, p.pulse_energy = s.get("t_center", 0.0), s.get("energy", 0.0)
    p.pulse_y0, p.pulse_z0 = s.get("y0", 0.0), s.get("z0", 0.0)
    p.init_dT = s.get("dT", 0.0)
    p.init_x_lo, p.init_x_hi = s.get("x_lo", 0.0), s.get("x_hi", 0.0)
    p.n_particles, p.seed, p.instance_id = r["n_particles"], r["seed"], r.get("instance_id", 0)
    p.max_scatter, p.max_events = r.get("max_scatter", 0), r.get("max_events", 1 << 20)
    p.max_collisions = r.get("max_collisions", 0)
    p.n_bins_x, p.n_batch = r.get("n_bins_x", 0), r.get("n_batch", 32)
    gx, gy, gz = r.get("grid", (0, 0, 0))
    p.grid_nx, p.grid_ny, p.grid_nz = gx, gy, gz
    p.n_samples = r.get("n_samples", 0)
    p.n_hj = r.get("n_hj", 0)
    p.t_final, p.sample_dt = r.get("t_final", 0.0), r.get("sample_dt", 0.0)
    p.n_threads = n_threads if n_threads else (os.cpu_count() or 1)
    p.record_particles = 1 if record_particles else 0
    my, mz = r.get("map", (0, 0))
    p.map_ny, p.map_nz = int(my), int(mz)
    return p


def run(prob, n_threads=None, record_particles=False, library=None):
    """Trace ``prob["run"]["n_particles"]`` particles; returns a dict of
    scalars, counters and (when requested by the problem) profile, H_j and
    transient-grid arrays, plus per-particle records when asked."""
    L = library if library is not None else lib()
    p = to_problem(prob, n_threads, record_particles)
    res = Result()
    nb, nh = max(p.n_bins_x, 0), max(p.n_hj, 0)
    T_mean, T_se, q_mean, q_se = (np.zeros(nb) for _ in range(4))
    h_mean, h_se = np.zeros(nh), np.zeros(nh)
    ncell = p.n_samples * p.grid_nx * p.grid_ny * p.grid_nz if p.n_samples > 0 else 0
    grid = np.zeros(ncell, dtype=np.int64)
    recs = np.zeros(p.n_particles if record_particles else 0, dtype=PARTICLE_DTYPE)
    nmap = p.map_ny * p.map_nz if p.map_ny > 0 and p.map_nz > 0 else 0
    maps = np.zeros(5 * nmap)

    def ptr(a):
        return a.ctypes.data if a.size else None

    rc = L.orc_run(C.byref(p), C.byref(res), ptr(T_mean), ptr(T_se), ptr(q_mean), ptr(q_se),
                   ptr(h_mean), ptr(h_se), ptr(grid), ptr(recs), ptr(maps))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (rc={rc})")
    out = {f[0]: getattr(res, f[0]) for f in Result._fields_}
    if nb:
        out.update(T=T_mean, T_se=T_se, q=q_mean, q_se=q_se)
    if nh:
        out.update(H=h_mean, H_se=h_se)
    if ncell:
        out["grid"] = grid.reshape(p.n_samples, p.grid_nz, p.grid_ny, p.grid_nx)
    if nmap:
        m = maps.reshape(5, p.map_nz, p.map_ny)
        out.update(map_T=m[0], map_T_se=m[1], map_q=m[2], map_q_se=m[3], map_solid=m[4])
    if record_particles:
        out["particles_rec"] = recs
    return out


def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(o)


def material(prob):
    """(omega, v, tau, C) per mode, FP64, as the oracle builds them."""
    p = to_problem(prob)
    n = lib().orc_material(C.byref(p), None, None, None, None, 0)
    if n < 0:
        raise ValueError("bad material")
    arrs = [np.zeros(n) for _ in range(4)]
    lib().orc_material(C.byref(p), *[a.ctypes.data for a in arrs], n)
    return tuple(arrs)


def draw_modes(prob, which, u):
    """Inverse-CDF mode draws for uniforms ``u``: which = 'emit', 'scatter' or 'initial'."""
    p = to_problem(prob)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(u.size, dtype=np.int32)
    code = {"emit": 0, "scatter": 1, "initial": 2}[which]
    rc = lib().orc_draw_modes(C.byref(p), code, u.ctypes.data, u.size,
                              out.ctypes.data)
    if rc:
        raise ValueError("bad material")
    return out


def scatter_direction(g, incoming, u_mu, u_phi):
    """Direction after a relaxation event (isotropic for g = 0, else the
    Henyey-Greenstein law of mean cosine g about ``incoming``)."""
    lib()
    inc = np.ascontiguousarray(incoming, dtype=np.float64)
    out = np.zeros(3)
    _lib.orc_scatter_direction(float(g), inc.ctypes.data, float(u_mu), float(u_phi), out.ctypes.data)
    return out


def first_boundary(prob, pos, direction):
    """Distance along the unit direction to the first boundary and its kind
    (0 none, 1 x=0, 2 x=L, 3 pore, 4 y=0, 5 y=pitch, 6 z=0, 7 z=pitch)."""
    p = to_problem(prob)
    a = np.ascontiguousarray(pos, dtype=np.float64)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    k = C.c_int32()
    t = lib().orc_first_boundary(C.byref(p), a.ctypes.data, d.ctypes.data, C.byref(k))
    return t, k.value


def emit(prob, first, n, library=None):
    """Initial states of particles first..first+n-1: columns (sign, x, y, z,
    ox, oy, oz, t0) and the mode ids."""
    p = to_problem(prob)
    out = np.zeros((n, 8))
    modes = np.zeros(n, dtype=np.int32)
    L = library if library is not None else lib()
    rc = L.orc_emit(C.byref(p), first, n, out.ctypes.data, modes.ctypes.data)
    if rc:
        raise ValueError("oracle rejected the problem")
    return out, modes
