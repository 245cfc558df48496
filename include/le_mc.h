/*
 * le_mc.h -- C ABI of the GB300 (sm_103a) trajectory tracer for the
 * linearized energy-based deviational Monte Carlo method (Peraud and
 * Hadjiconstantinou, "An alternative approach to efficient simulation of
 * micro/nanoscale phonon transport", arXiv:1206.3316).
 *
 * Under the linearized collision operator (Eq. 2) deviational particles do
 * not interact, so each trajectory is traced alone from emission to
 * termination (trajectory algorithm, steps I-VI) and contributes to
 * path-integrated (Eq. 4) or time-sampled (Eq. 3) estimators.  This library
 * runs that loop on one GPU.
 *
 * Conventions for every function below:
 *  - All functions return an le_mc_status; none aborts, exits or prints.
 *    A failed call leaves a thread-local message in le_mc_last_error().
 *  - Pointers are HOST pointers unless a comment says "device pointer".
 *    Descriptors are read during the call only; the caller keeps ownership.
 *  - Handles are opaque and owned by the caller until the matching destroy.
 *    Materials and geometries are immutable after creation and may be used
 *    by any number of runs, including concurrent ones; the library keeps them
 *    alive (reference count) until the last run using them is destroyed.
 *  - Device memory is allocated by the library from the stream-ordered pool
 *    of the current device; results are copied into caller-owned buffers.
 *  - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).
 *  - SI units (m, s, K, J, W) throughout; the gray material may be
 *    non-dimensional as long as it is used consistently.
 */
#ifndef LE_MC_H
#define LE_MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LE_MC_API __attribute__((visibility("default")))
#else
#define LE_MC_API
#endif

#define LE_MC_ABI_VERSION 5
#define LE_MC_MAX_BRANCHES 4
#define LE_MC_MAX_MODES 4096        /* mode tables live in shared memory       */
#define LE_MC_MAX_BINS_X 256        /* slab profile bins                       */
#define LE_MC_MAX_BATCH 64          /* batch groups for profile error bars     */
#define LE_MC_MAX_HJ 128            /* per-scattering-index flux tallies       */
#define LE_MC_MAX_MAP 64            /* steady map cells per axis               */

/* Bits of le_mc_tallies.device_flags, set on the device (never a trap):
 * REJECTION_EXHAUSTED: a rejection loop of step I (positions outside the
 *   pores, pulse times >= 0) used all its 64 tries; that particle starts from
 *   its last draw.
 * BAD_LAUNCH: a trace kernel found a launch shape it cannot run (threads per
 *   block not a multiple of 32, or above 512) and traced nothing; the entry
 *   points validate shapes first, so this marks a library defect. */
#define LE_MC_FLAG_REJECTION_EXHAUSTED 1u
#define LE_MC_FLAG_BAD_LAUNCH 4u
/* DEBUG_BOUNDS (debug builds, -DLEMC_DEBUG, only): a data-dependent index of
 * a trace kernel (emission-buffer slot, mode, queue position, batch
 * instance, sample-job owner, record slot) was out of range and its access was
 * redirected to index 0, or a transient cell, slab-profile bin or map cell
 * was computed more than one cell outside its grid. */
#define LE_MC_FLAG_DEBUG_BOUNDS 8u

typedef enum {
    LE_MC_OK = 0,
    LE_MC_ERR_INVALID = 1, /* a descriptor field or argument is out of range     */
    LE_MC_ERR_NOMEM = 2,   /* a host or device allocation failed                 */
    LE_MC_ERR_CUDA = 3,    /* a CUDA runtime call failed                         */
    LE_MC_ERR_TIMEOUT = 4, /* a bounded wait ended first (le_mc_server_wait_all) */
    LE_MC_ERR_BUDGET = 5,  /* reserved: no entry point returns it at present      */
    LE_MC_ERR_STATE = 6,   /* the handle is unusable (earlier failure) or busy    */
    LE_MC_ERR_NODEV = 7    /* no usable CUDA device                              */
} le_mc_status;

/* ---- material (Eq. 1 ingredients at the control temperature T_eq) ---------
 * Per mode b (branch p, frequency bin): C_b = g_p D_p(w_b) hbar w_b
 * d f_BE/dT(w_b, T_eq) dw (J m^-3 K^-1), group velocity v_b, relaxation time
 * tau_b = tau(w_b, p, T_eq) (material properties at T_0, as in the linear
 * regime paragraph after Eq. 5), mean free path Lambda_b = v_b tau_b.       */
enum { LE_MC_MAT_GRAY = 0, LE_MC_MAT_QUADRATIC = 1, LE_MC_MAT_TABULATED = 2 };

typedef struct {
    int32_t kind;          /* LE_MC_MAT_*                                        */
    int32_t n_branch;      /* QUADRATIC: number of branches, 1..4                */
    int32_t n_bins;        /* QUADRATIC: equal-width frequency bins per branch   */
    int32_t n_modes;       /* TABULATED: number of modes, 1..LE_MC_MAX_MODES     */
    double T_eq;           /* control temperature [K] (> 0)                      */
    double gray_v, gray_tau, gray_C; /* GRAY: one mode                           */
    /* QUADRATIC: omega(k) = c1 k + c2 k^2 per branch, degeneracy g_p, k up to
     * min(2 pi / a_lattice, c1 / (2|c2|)) (the group velocity stays > 0),
     * 1/tau = A omega^4 + B omega^2 T exp(-C_exp / T) for every branch.         */
    double c1[LE_MC_MAX_BRANCHES], c2[LE_MC_MAX_BRANCHES], degeneracy[LE_MC_MAX_BRANCHES];
    double a_lattice, A, B, C_exp;
    /* TABULATED: host arrays of n_modes values (copied during the call)        */
    const double* tab_v;
    const double* tab_tau;
    const double* tab_C;
    /* Direction change at a relaxation event (step IVb): 0 keeps the paper's
     * isotropic redraw; a nonzero g in (-1, 1) draws the new direction from
     * the Henyey-Greenstein law of mean cosine g about the incoming one (the
     * generalisation the paper allows; the mode is still redrawn from the
     * normalised Eq. 2, independently of the direction).                     */
    double scatter_g;
} le_mc_material_desc;

typedef struct le_mc_material_s* le_mc_material;

/* Builds the per-mode tables in FP64 on the host, the alias tables of the
 * emission law (weights C_b v_b: boundary source after the algorithm, Eq. 6)
 * and of the post-scattering law (weights C_b / tau_b: normalised Eq. 2), and
 * uploads them to the current device.  Synchronous.
 * Errors: LE_MC_ERR_INVALID (bad field, zero total weight, > MAX_MODES),
 * LE_MC_ERR_NOMEM, LE_MC_ERR_CUDA, LE_MC_ERR_NODEV. */
LE_MC_API le_mc_status le_mc_create_material(const le_mc_material_desc* desc, le_mc_material* out);
LE_MC_API le_mc_status le_mc_destroy_material(le_mc_material m);

/* Host-only: the FP64 mode table the material would hold, without touching a
 * GPU.  Arrays of `capacity` doubles (NULL to query); *n_modes receives the
 * count.  Errors: LE_MC_ERR_INVALID. */
LE_MC_API le_mc_status le_mc_material_table(const le_mc_material_desc* desc, double* omega, double* v,
                                  double* tau, double* C, int32_t capacity, int32_t* n_modes);

/* Host-only: Vose alias table of n weights (n <= LE_MC_MAX_MODES) in the
 * library's sampling format: a draw of a uniform 32-bit word r picks column
 * j = floor(r n / 2^32) and returns j if (r n mod 2^32) < threshold[j], else
 * alias[j].  Errors: LE_MC_ERR_INVALID (n out of range, negative or all-zero
 * weights). */
LE_MC_API le_mc_status le_mc_alias_table(const double* weights, int32_t n, uint32_t* threshold, uint32_t* alias);

/* ---- geometry (step III boundary search, step IVa wall response) --------- */
enum { LE_MC_GEOM_PLANES = 0, LE_MC_GEOM_BULK = 1, LE_MC_GEOM_POROUS = 2 };
/* Wall laws (step IVa): BLACK absorbs (isothermal wall, the particle ends);
 * DIFFUSE re-emits with a cosine law about the inward normal, mode kept;
 * SPECULAR mirrors the direction; PARTIAL is specular with probability
 * spec_* and diffuse otherwise (the choice uses the flight's second uniform,
 * which only a relaxation event uses otherwise). */
enum { LE_MC_WALL_BLACK = 0, LE_MC_WALL_DIFFUSE = 1, LE_MC_WALL_SPECULAR = 2, LE_MC_WALL_PARTIAL = 3 };

typedef struct {
    int32_t kind;      /* PLANES: walls at x = 0 and x = L, unbounded in y, z (slab, film)
                        * BULK:   no boundaries
                        * POROUS: PLANES plus cylindrical pores along x centred in
                        *         each pitch x pitch unit cell of the (y, z) plane;
                        *         the domain is cells_y x cells_z unit cells,
                        *         periodic in y and z (particles crossing a face are
                        *         re-inserted on the opposite face)               */
    int32_t wall_lo;   /* wall type at x = 0 (LE_MC_WALL_*)                     */
    int32_t wall_hi;   /* wall type at x = L                                   */
    int32_t pore_wall; /* POROUS: pore surface type (DIFFUSE, SPECULAR, PARTIAL) */
    double L;          /* thickness along x [m] (> 0 unless BULK)               */
    double pitch;      /* POROUS: lattice pitch [m]                            */
    double radius;     /* POROUS: pore radius [m], 0 <= 2 radius < pitch         */
    int32_t cells_y, cells_z; /* POROUS: periodic domain in unit cells (>= 1)   */
    double spec_lo, spec_hi;  /* PARTIAL walls at x = 0, x = L: probability of a
                               * specular reflection, in [0, 1]               */
    double spec_pore;         /* PARTIAL pore surface: the same               */
} le_mc_geometry_desc;

typedef struct le_mc_geometry_s* le_mc_geometry;

/* Validates and stores the geometry.  Errors: LE_MC_ERR_INVALID. */
LE_MC_API le_mc_status le_mc_create_geometry(const le_mc_geometry_desc* desc, le_mc_geometry* out);

/* Host-only: solid fraction of each cell of a map_ny x map_nz map over the
 * (y, z) unit cell of a POROUS geometry (the cell minus its overlap with the
 * pore's circle, exact), written to fraction[map_nz][map_ny].  These are the
 * fractions that normalise the steady maps (LE_MC_ARRAY_MAP_SOLID).
 * Errors: LE_MC_ERR_INVALID (not POROUS, sizes out of 1..LE_MC_MAX_MAP). */
LE_MC_API le_mc_status le_mc_map_solid(const le_mc_geometry_desc* g, int32_t map_ny, int32_t map_nz, double* fraction);

LE_MC_API le_mc_status le_mc_destroy_geometry(le_mc_geometry g);

/* ---- run: sources (step I), termination (step VI), estimators (step V) ---- */
enum { LE_MC_SRC_WALLS = 0, LE_MC_SRC_GRADIENT = 1, LE_MC_SRC_PULSE = 2, LE_MC_SRC_INITIAL = 3 };
enum { LE_MC_PREC_FP64 = 0, LE_MC_PREC_FP32 = 1 };

typedef struct {
    int32_t source;    /* WALLS (PLANES only): isothermal walls at T_eq + dT_lo
                        *   (x = 0) and T_eq + dT_hi (x = L) emit V_g cos C |dT|
                        *   into the domain; black walls absorb (boundary source
                        *   after the algorithm).
                        * GRADIENT: the volumetric source of Eq. 5 / Eq. 6 for a
                        *   uniform dT/dz, equal numbers of each sign.
                        * PULSE (POROUS only): surface heat pulse on x = L,
                        *   Gaussian in (y, z) and in time, all signs positive.
                        * INITIAL (POROUS only): initial condition
                        *   C_{w,p} |T_i - T_eq| delta(t) of the text after the
                        *   algorithm: a uniform excess init_dT in the layer
                        *   init_x_lo < x < init_x_hi at t = 0, modes weighted
                        *   by C_b, isotropic directions.                       */
    int32_t precision; /* FP64: every step in FP64.  FP32: trajectory geometry and
                        *   times in FP32, per-particle sums carried compensated,
                        *   tally accumulation in FP64.                          */
    double dT_lo, dT_hi;            /* WALLS [K]                                  */
    double dTdz;                    /* GRADIENT [K/m], nonzero                    */
    double pulse_sigma_x;           /* PULSE: lateral standard deviation [m]     */
    double pulse_sigma_t;           /* PULSE: temporal standard deviation [s]    */
    double pulse_t_center;          /* PULSE: centre time [s] (times < 0 redrawn) */
    double pulse_energy;            /* PULSE: deviational energy [J]             */
    double pulse_y0, pulse_z0;      /* PULSE: centre in the periodic domain [m]  */
    uint64_t n_particles;           /* N, 0 .. 2^32 - 1 (2^31 - 1 for PULSE)     */
    uint64_t seed;                  /* Philox4x32-10 key                         */
    uint32_t instance_id;           /* 4th counter word: independent streams     */
    uint32_t max_scatter;           /* terminate at this scattering event (0 = none) */
    uint32_t max_events;            /* terminate after this many segments (>= 1) */
    int32_t n_bins_x;               /* profile bins along x (0 = off): WALLS,
                                     * T(x) and q_x(x); GRADIENT between planes,
                                     * T(x) and the in-plane flux q_z(x)        */
    int32_t n_batch;                /* batch groups of the error bars: slab
                                     * profiles group particle ids mod n_batch,
                                     * maps group particle pairs (2i, 2i + 1)
                                     * mod n_batch, so that every group holds
                                     * both signs of the gradient source        */
    int32_t grid_nx, grid_ny, grid_nz; /* PULSE, INITIAL: counting grid over the
                                        * L x domain                          */
    int32_t n_samples;              /* PULSE, INITIAL: sample times (k + 1/2)
                                     * sample_dt, k < n_samples <= 2^20        */
    double t_final;                 /* PULSE, INITIAL: end of the simulation [s] */
    double sample_dt;               /* PULSE, INITIAL: sample spacing [s]        */
    int32_t n_hj;                   /* flux split by scattering index j (0 = off;
                                     * steady sources only)                     */
    int32_t record_particles;       /* 1: keep one le_mc_particle per particle   */
    int32_t blocks_per_sm;          /* launch shape (0 = library default)        */
    int32_t threads_per_block;      /* 0 = default: 512, or 256 when that keeps more
                                     * warps resident; else a multiple of 32, <= 512 */
    int32_t schedule;               /* particle order: 0 auto, 1 long-first,
                                     * 2 natural id order.  Long-first serves
                                     * particles emitted in modes with a mean
                                     * free path above long_mfp_cut before the
                                     * rest, so the longest trajectories overlap
                                     * the bulk instead of trailing it.  Results
                                     * do not depend on the order (up to FP64
                                     * summation order).                       */
    int32_t refill_min;             /* a warp refills idle lanes once this many
                                     * are idle (0 = library default, 4)         */
    double long_mfp_cut;            /* [m]; 0 = 32 L (PLANES, POROUS).  Runs of
                                     * at most 2^25 particles also trace those
                                     * above 32 times this first, each by a warp
                                     * of its own (at most 512)                */
    int32_t chunk;                  /* queue positions a warp claims per atomic,
                                     * multiple of 32 (0 = library default, 256) */
    uint32_t first_particle;        /* particle ids traced are first_particle ..
                                     * first_particle + n_particles - 1 (< 2^32),
                                     * so a problem can be traced in pieces      */
    double init_dT;                 /* INITIAL: T_i - T_eq [K], nonzero          */
    double init_x_lo, init_x_hi;    /* INITIAL: heated layer, 0 <= lo < hi <= L  */
    uint32_t max_collisions;        /* terminate at this many relaxations + wall
                                     * hits, crossings of periodic unit-cell
                                     * faces not counted (0 = none); 1 follows
                                     * each particle over its first free path
                                     * only (the first-free-path estimate)     */
    int32_t map_ny, map_nz;         /* POROUS + GRADIENT: steady maps over the
                                     * (y, z) unit cell, integrated through the
                                     * thickness (Eq. 4 per map cell), on
                                     * map_ny x map_nz equal cells (0 = off;
                                     * 1..LE_MC_MAX_MAP each); error bars from
                                     * the n_batch groups                      */
} le_mc_run_desc;

typedef struct le_mc_run_s* le_mc_run_handle;

/* Enqueues one simulation on `stream` and returns at once: device tallies are
 * allocated and zeroed, the persistent trace kernel (steps I-VI with the
 * estimators of step V) is launched, and the run's completion is recorded.
 * The particle stream is fixed by (seed, instance_id, particle id), so the
 * tallies do not depend on the launch shape up to FP64 summation order.
 * Errors: LE_MC_ERR_INVALID (descriptor out of range or inconsistent with the
 * geometry), LE_MC_ERR_NOMEM, LE_MC_ERR_CUDA. */
LE_MC_API le_mc_status le_mc_run(le_mc_material m, le_mc_geometry g, const le_mc_run_desc* desc,
                       void* stream, le_mc_run_handle* out);

/* Blocks until the run's device work is complete.
 * Errors: LE_MC_ERR_INVALID (null handle), LE_MC_ERR_STATE (the run failed
 * earlier), LE_MC_ERR_CUDA (the device work failed; the handle then reports
 * LE_MC_ERR_STATE). */
LE_MC_API le_mc_status le_mc_wait(le_mc_run_handle h);

typedef struct {
    double P_total;     /* source power: W per m^2 of wall (WALLS), W over the solid
                         * part of the reference volume (GRADIENT)                */
    double E_eff_dot;   /* steady: effective deviational power per particle (Eq. 4) */
    double E_eff;       /* PULSE, INITIAL: deviational energy per particle (Eq. 3) */
    double C_tot;       /* sum_b C_b                                               */
    double sum_sL, sum_sL2; /* sum over particles of s L and (s L)^2, L the total
                             * algebraic length along the flux axis (x for WALLS,
                             * z otherwise)                                        */
    double flux, flux_se;   /* heat flux along that axis [W/m^2] and its std error  */
    double kappa, kappa_se; /* GRADIENT: -flux / (dT/dz)                           */
    double kappa_solid;     /* POROUS: flux averaged over the solid only           */
    double psi, psi_se;     /* WALLS: flux / (sum_b C_b v_b / 4 (dT_lo - dT_hi))   */
    uint64_t particles, segments, scatters, wall_hits, periodic, truncated, absorbed;
    double kernel_ms;       /* device time of the trace kernel                    */
    double prepass_ms;      /* device time of the long-first classification pass  */
    uint32_t kernel_launches; /* kernels this run launched                        */
    uint32_t device_flags;  /* device-side status bits, LE_MC_FLAG_* (0 = none)  */
    uint32_t long_listed;   /* particles served from the long-first list (their
                             * emission mean free path above long_mfp_cut)    */
    uint32_t extreme_traced; /* particles traced apart, one per warp whose idle
                             * lanes precompute its random words (above 32 x
                             * long_mfp_cut; 0 when more than the list holds) */
} le_mc_tallies;

/* Waits for the run, copies the tallies to the host and normalises them
 * (N = energy / E_eff after the algorithm; Eq. 4 for steady runs).
 * Errors: LE_MC_ERR_STATE (failed run), LE_MC_ERR_CUDA. */
LE_MC_API le_mc_status le_mc_read_tallies(le_mc_run_handle h, le_mc_tallies* out);

/* Arrays of a finished run, copied into caller memory of `capacity` bytes
 * (*written receives the byte count; call with dst = NULL to query it):
 *   T, T_SE, Q, Q_SE : double[n_bins_x]  temperature T - T_eq (energy
 *                      temperature) of each slab along x and the heat flux
 *                      there along the flux axis (x for WALLS; z for
 *                      GRADIENT: the in-plane flux of a film by depth), with
 *                      batch-mean errors
 *   H, H_SE          : double[n_hj]      flux carried between scattering
 *                      events j and j+1 (j = 0: emission to first scattering)
 *   GRID             : int32[n_samples][grid_nz][grid_ny][grid_nx] signed
 *                      particle counts of Eq. 3 (times E_eff = energy per cell)
 *   PARTICLES        : le_mc_particle[n_particles] (record_particles = 1)
 *   GRID_T           : double[n_samples][grid_nz][grid_ny][grid_nx]  energy
 *                      temperature T - T_eq of each cell at each sample time
 *                      (Eq. 3 count times E_eff / (C_tot V_cell), V_cell the
 *                      whole cell, pores included)
 *   GRID_TX          : double[n_samples][grid_nx]  T - T_eq averaged over the
 *                      solid of each x slab (the pores run through the whole
 *                      thickness, so every slab holds the same solid volume):
 *                      the temperature history of a layer, as a
 *                      thermoreflectance-like transient reads it
 *   GRID_T_SE, GRID_TX_SE : double, shaped as GRID_T and GRID_TX: standard
 *                      errors of those values.  A particle is in at most one
 *                      cell (one slab) at a sample time and all particles of
 *                      the transient sources carry one sign, so a count n of
 *                      N particles has the estimated variance
 *                      N/(N-1) |n| (1 - |n|/N)
 *   MAP_T, MAP_T_SE   : double[map_nz][map_ny]  steady T - T_eq(z) over the
 *                      solid of each map cell (time-integrated deviational
 *                      energy over C_tot x solid volume; add the imposed
 *                      linear T_eq(z) for the local temperature), and its
 *                      batch-means standard error; NaN where a cell holds
 *                      no solid
 *   MAP_Q, MAP_Q_SE   : double[map_nz][map_ny]  local heat flux along z over
 *                      the solid of each map cell [W/m^2] and its standard
 *                      error; NaN where a cell holds no solid
 *   MAP_SOLID         : double[map_nz][map_ny]  solid fraction of each map
 *                      cell (exact, from the pore's circle)
 *   MAP_T_LOCAL       : double[map_nz][map_ny]  local temperature T - T_0 of
 *                      each map cell: MAP_T plus the imposed linear T_eq(z) -
 *                      T_0 = (z - pitch/2) dT/dz at the cell's centre (T_0 the
 *                      control temperature, reached at the unit cell's mid-
 *                      plane z = pitch/2); NaN where a cell holds no solid
 * Errors: LE_MC_ERR_INVALID (array not produced by this run, capacity too
 * small), LE_MC_ERR_STATE, LE_MC_ERR_CUDA. */
enum { LE_MC_ARRAY_T = 0, LE_MC_ARRAY_T_SE = 1, LE_MC_ARRAY_Q = 2, LE_MC_ARRAY_Q_SE = 3,
       LE_MC_ARRAY_H = 4, LE_MC_ARRAY_H_SE = 5, LE_MC_ARRAY_GRID = 6, LE_MC_ARRAY_PARTICLES = 7,
       LE_MC_ARRAY_GRID_T = 8, LE_MC_ARRAY_GRID_TX = 9, LE_MC_ARRAY_GRID_T_SE = 10, LE_MC_ARRAY_GRID_TX_SE = 11,
       LE_MC_ARRAY_MAP_T = 12, LE_MC_ARRAY_MAP_T_SE = 13, LE_MC_ARRAY_MAP_Q = 14, LE_MC_ARRAY_MAP_Q_SE = 15,
       LE_MC_ARRAY_MAP_SOLID = 16, LE_MC_ARRAY_MAP_T_LOCAL = 17 };
LE_MC_API le_mc_status le_mc_read_array(le_mc_run_handle h, int32_t which, void* dst, size_t capacity,
                              size_t* written);

typedef struct {
    int8_t sign;        /* +1 / -1                                                 */
    int8_t fate;        /* 0 absorbed, 1 scattering cap, 2 segment cap, 3 t_final,
                         * 4 collision cap (max_collisions)                        */
    int16_t pad;
    uint32_t n_seg, n_scat, n_wall, n_periodic;
    uint32_t mode0;     /* emitted mode                                            */
    double L_axis;      /* algebraic length along the flux axis                    */
    double x0, t0;      /* emission position along x and emission time             */
} le_mc_particle;

LE_MC_API le_mc_status le_mc_destroy_run(le_mc_run_handle h);

/* ---- choosing the scattering cap K_s from the flux split -------------------
 * The paper truncates histories of non-absorbing domains after about 40
 * relaxation events, chosen where the flux carried between the j-th and
 * (j+1)-th relaxation, <H_j>, becomes of the order of its own statistical
 * uncertainty; it notes that <H_j> decays exponentially, which keeps the
 * error of the cap under control (termination discussion after Eq. 4, its
 * Fig. 2 c-d).  This host-only study reads the H / H_se arrays of a run with
 * n_hj > 0 (LE_MC_ARRAY_H, LE_MC_ARRAY_H_SE):
 *   k_s    the first j with |<H_j>| <= its standard error (n if none);
 *   ratio, amp, sign: the geometric law sign amp ratio^j fitted by weighted
 *          least squares on log |<H_j>| (weights (H_j / se_j)^2) over the
 *          contiguous run of indices from `first` on whose |<H_j>| exceeds
 *          `resolved` standard errors (ratio = NaN if fewer than n_fit = 2);
 * and le_mc_truncation_tail gives the flux a cap K drops, the extrapolated
 * sum_{j >= K} <H_j> = sign amp ratio^K / (1 - ratio) (0 unless 0 < ratio
 * < 1).  Errors: LE_MC_ERR_INVALID (null pointer, n out of 1..LE_MC_MAX_HJ,
 * resolved <= 0, first < 0, a non-finite H or negative H_se). */
typedef struct {
    int32_t k_s;        /* first j with |H_j| <= H_se_j                     */
    int32_t n_fit;      /* indices in the fitted run                        */
    double ratio;       /* decay ratio of |H_j| per relaxation (NaN: no fit) */
    double amp;         /* |H_j| ~ amp ratio^j                              */
    double sign;        /* sign of the fitted terms' sum                    */
} le_mc_truncation;
LE_MC_API le_mc_status le_mc_truncation_study(const double* H, const double* H_se, int32_t n, double resolved,
                                              int32_t first, le_mc_truncation* out);
/* Extrapolated flux dropped by a cap at K relaxations (K >= 0) from a study;
 * host-only.  Errors: LE_MC_ERR_INVALID (null pointer, K < 0). */
LE_MC_API le_mc_status le_mc_truncation_tail(const le_mc_truncation* study, int32_t K, double* dropped);

/* ---- batches: many instances of one problem family in one launch ---------
 * Not in the paper: the instances are independent simulations of the method
 * (same steps I-VI), packed into one persistent launch so that small
 * instances do not leave the GPU idle.  The particle stream of an instance is
 * fixed by (seed, instance_id, particle id), so each instance's result is the
 * one le_mc_run gives for it alone, up to FP64 summation order. */
typedef struct le_mc_batch_s* le_mc_batch;

typedef struct {
    int32_t threads_per_block; /* 0 = 512                                   */
    int32_t blocks_per_sm;     /* 0 = as many as fit                        */
    int32_t refill_min;        /* 0 = 1                                     */
    int32_t chunk;             /* queue positions per claim, 0 = 32         */
    int32_t use_graph;         /* 1: capture zero + classify + trace once as
                                * a CUDA graph and replay it per launch     */
    float ms;                  /* autotune: time of one launch with this shape */
} le_mc_launch_config;

/* n >= 1 instances sharing material m.  All geoms[i] are PLANES with the same
 * wall types; all runs[i] share source kind, precision, seed, max_scatter and
 * max_events; each has its own thickness geoms[i].L, drive (dT_lo, dT_hi or
 * dTdz), n_particles and instance_id.  Profiles, H_j, grids and records are
 * not available in batches.  The sum of n_particles must be < 2^32.  Device
 * memory for every instance's tallies is allocated here, once.
 * Errors: LE_MC_ERR_INVALID, LE_MC_ERR_NOMEM, LE_MC_ERR_CUDA. */
LE_MC_API le_mc_status le_mc_batch_create(le_mc_material m, int32_t n, const le_mc_geometry_desc* geoms,
                                          const le_mc_run_desc* runs, le_mc_batch* out);
/* Launch shape of later launches (drops a captured graph).  INVALID if out of range. */
LE_MC_API le_mc_status le_mc_batch_set_config(le_mc_batch b, const le_mc_launch_config* cfg);
/* Enqueues one pass over every instance on `stream`: zero the tallies,
 * classify (long-first), trace.  Asynchronous; a launch may overlap nothing
 * else that uses the same batch. */
LE_MC_API le_mc_status le_mc_batch_launch(le_mc_batch b, void* stream);
LE_MC_API le_mc_status le_mc_batch_wait(le_mc_batch b);
/* Tallies of instance i from the last launch (waits for it); kernel_ms is the
 * device time of the whole launch. */
LE_MC_API le_mc_status le_mc_batch_read(le_mc_batch b, int32_t i, le_mc_tallies* out);
/* Picks threads_per_block, blocks_per_sm, refill_min and chunk by timing
 * launches of this batch (each candidate once after one warm-up), sets the
 * best and returns it.  If cache_path is not NULL, a previous result for the
 * same (geometry kind, source, precision, mode count, GPU name) is reused and
 * a new one appended.  Synchronous on `stream`. */
LE_MC_API le_mc_status le_mc_batch_autotune(le_mc_batch b, void* stream, const char* cache_path,
                                            le_mc_launch_config* best);
LE_MC_API le_mc_status le_mc_batch_destroy(le_mc_batch b);

/* ---- serving: continuous batching of simulation requests -------------------
 * Not in the paper.  A worker thread owned by the server admits submitted
 * requests into slots while a slot and device memory are free.  An admitted
 * request's parameters, tables and running tallies stay in device memory
 * until it retires.  Its particles are traced in epochs over consecutive
 * particle-id ranges; each epoch is published as work items to a ring that
 * one resident persistent kernel drains, so the particles of every admitted
 * request (slabs, films, pored films and bulk, each with its own material)
 * are interleaved inside that kernel.  The kernel leaves on its own after
 * idle_exit_ms without work and is launched again when work arrives.  A
 * request retires once the relative standard error of its primary estimate
 * (kappa for GRADIENT, Psi for WALLS) is at or below its target, or its
 * particle budget is spent.  A request's epoch sizes depend only on its own
 * statistics, so its particle set, and therefore its result, is the same
 * whether it runs alone or among others (up to FP64 summation order).
 * Served requests: steady WALLS (PLANES) or GRADIENT sources, FP32
 * trajectories, isotropic relaxation events, black, diffuse or specular
 * walls and pores, no arrays. */
typedef struct le_mc_server_s* le_mc_server;

typedef struct {
    int32_t max_slots;             /* requests traced at once, 1..64 (0 = 8)        */
    int32_t pad;
    uint64_t hbm_budget_bytes;     /* device memory active requests may hold
                                    * (0 = half of the free memory at creation)    */
    uint64_t pilot_particles;      /* first epoch of every request (0 = 65536)      */
    uint64_t max_epoch_particles;  /* largest epoch of one request (0 = 2^24)       */
    int32_t idle_exit_ms;          /* the resident kernel leaves after this long
                                    * without work, 0..60000 (0 = 250)            */
    int32_t pad2;
} le_mc_server_config;

enum { LE_MC_REQ_QUEUED = 0, LE_MC_REQ_RUNNING = 1, LE_MC_REQ_DONE = 2, LE_MC_REQ_FAILED = 3 };

typedef struct {
    int32_t state;                 /* LE_MC_REQ_*                                   */
    int32_t epochs;                /* epochs traced for the request                 */
    double submit_s, start_s, done_s; /* server clock, seconds since creation        */
    double rel_err;                /* achieved relative std error of the estimate   */
    le_mc_tallies tallies;         /* over every particle traced for the request    */
} le_mc_request_status;

typedef struct {
    uint64_t submitted, completed, failed, active, queued;
    uint64_t segments, particles;  /* traced by completed epochs                    */
    uint64_t hbm_in_use;           /* bytes held by admitted requests (estimate)    */
    double uptime_s;
    uint64_t kernel_launches;      /* launches of the resident kernel so far         */
} le_mc_server_counters;

/* Starts the worker thread on the current device.  Errors: INVALID, NOMEM, CUDA. */
LE_MC_API le_mc_status le_mc_server_create(const le_mc_server_config* cfg, le_mc_server* out);
/* Queues a request; r->n_particles is its particle budget, target_rel_err > 0
 * its goal.  Descriptors are copied.  WALLS or GRADIENT sources only.
 * Errors: INVALID (descriptor or target), STATE (server stopping). */
LE_MC_API le_mc_status le_mc_server_submit(le_mc_server s, const le_mc_material_desc* m,
                                           const le_mc_geometry_desc* g, const le_mc_run_desc* r,
                                           double target_rel_err, uint64_t* request_id);
/* Non-blocking status of a request.  Errors: INVALID (unknown id). */
LE_MC_API le_mc_status le_mc_server_poll(le_mc_server s, uint64_t request_id, le_mc_request_status* out);
/* A queued request fails at once; a running one after its epoch in flight. */
LE_MC_API le_mc_status le_mc_server_cancel(le_mc_server s, uint64_t request_id);
/* Blocks until no request is queued or running; TIMEOUT after timeout_s. */
LE_MC_API le_mc_status le_mc_server_wait_all(le_mc_server s, double timeout_s);
LE_MC_API le_mc_status le_mc_server_stats(le_mc_server s, le_mc_server_counters* out);
/* Cancels what is queued, lets epochs in flight finish, joins the worker. */
LE_MC_API le_mc_status le_mc_server_destroy(le_mc_server s);

/* ---- tracing without allocation -------------------------------------------
 * The paper has no counterpart: this is a service for callers that must not
 * allocate GPU memory while they trace, e.g. code running inside a host
 * callback or in a region whose device memory belongs to a framework's own
 * allocator (a cudaMalloc there fails, blocks, or corrupts the allocator's
 * accounting), or a loop that cannot pay for an allocator call.  They create
 * the material and geometry beforehand and pass their own result buffers.
 *
 * le_mc_run_noalloc traces particles first_particle .. first_particle +
 * n_particles - 1 exactly like le_mc_run and writes the raw results to the
 * caller's DEVICE buffers: d_sums[2] = (sum s L, sum (s L)^2) over particles
 * (doubles) and d_counters[7] = (particles, segments, scatterings, wall
 * hits, periodic crossings, truncated, absorbed) (unsigned 64-bit); both are
 * cleared first.  It calls no cudaMalloc, cudaMallocAsync, cudaFree or
 * allocating library routine and creates no stream or event.  Its kernel
 * scratch (queue head, flags, long-first list and bitmap) is one fixed
 * device array inside the library, about 0.6 MB, held by every GPU that
 * loads the library until the process exits; that is why n_particles is
 * limited to LE_MC_NOALLOC_MAX_PARTICLES per call (larger problems are
 * traced in pieces with first_particle and the caller adds the pieces).
 * The array's device address is looked up during the first call on each
 * device, so make that first call before any stream capture; the address is
 * kept for the life of the process, so do not use the library across a
 * cudaDeviceReset.  Every call shares the array: calls whose device work
 * overlaps in time race on it, so the caller must serialise them.  Steady
 * WALLS / GRADIENT runs only (no profiles, maps, H_j, grid or records).
 * Asynchronous on `stream`.
 * Lifetime: the call takes no reference on the material, so the material
 * must outlive the call's device work; le_mc_destroy_material on a material
 * this entry point has used waits for the whole device before it frees the
 * tables, which makes an early destroy safe but costs a device-wide
 * synchronisation.
 * Device status bits (LE_MC_FLAG_*, e.g. REJECTION_EXHAUSTED from a pored
 * film's position draws) are not part of d_sums / d_counters; they stay in
 * the library's array until the next call and are read with
 * le_mc_noalloc_flags.
 * Errors: LE_MC_ERR_INVALID (null pointer, bad descriptor, n_particles above
 * the limit, arrays requested), LE_MC_ERR_CUDA. */
#define LE_MC_NOALLOC_MAX_PARTICLES (1u << 22)
LE_MC_API le_mc_status le_mc_run_noalloc(le_mc_material m, le_mc_geometry g, const le_mc_run_desc* desc,
                                         double* d_sums, unsigned long long* d_counters, void* stream);
/* Device status bits (LE_MC_FLAG_*) of the last le_mc_run_noalloc call on the
 * current device, copied into *flags once `stream` (the stream of that call)
 * has finished its work.  Synchronous; allocates nothing.
 * Errors: LE_MC_ERR_INVALID (null flags), LE_MC_ERR_CUDA. */
LE_MC_API le_mc_status le_mc_noalloc_flags(void* stream, uint32_t* flags);

/* ---- diagnostics ---------------------------------------------------------- */
/* Philox4x32-10 of n counters (4 words each) under one key, computed by a GPU
 * kernel; host arrays in and out.  Synchronous. */
LE_MC_API le_mc_status le_mc_philox(const uint32_t* counters, uint32_t key0, uint32_t key1, uint32_t* out,
                          size_t n);

/* Mode draws of the device alias tables (which = 0 emission, 1 scattering)
 * for n uniform 32-bit words; host arrays.  Synchronous. */
LE_MC_API le_mc_status le_mc_sample_modes(le_mc_material m, int32_t which, const uint32_t* words,
                                int32_t* modes, size_t n);

/* Current device: SM count and name (NULL-safe). */
LE_MC_API le_mc_status le_mc_device_info(int32_t* sm_count, char* name, size_t name_capacity);

/* sizeof of the ABI structs, for binding checks: which = 0 material_desc,
 * 1 geometry_desc, 2 run_desc, 3 tallies, 4 particle, 5 launch_config;
 * -1 if unknown. */
LE_MC_API int32_t le_mc_struct_size(int32_t which);

/* Thread-local description of the last failure on this thread ("" if none). */
LE_MC_API const char* le_mc_last_error(void);
/* LE_MC_ABI_VERSION of the built library. */
LE_MC_API int32_t le_mc_abi_version(void);

/* Test hook for failure handling: the after-th next device allocation made by
 * the library for a material, a run or a batch (0 = the very next one)
 * reports out of memory, so the caller sees LE_MC_ERR_NOMEM from that call
 * with nothing leaked; the hook then disarms itself.  after < 0 disarms it.
 * Process-wide.  Errors: none. */
LE_MC_API le_mc_status le_mc_test_fail_allocation(int32_t after);

#ifdef __cplusplus
}
#endif
#endif /* LE_MC_H */
