// Persistent trajectory kernel of the le_mc library: steps I-VI of the
// paper's trajectory algorithm for independent deviational particles, with
// the estimators of step V (Eq. 3 time samples, Eq. 4 path integrals).
//
// Work distribution.  Each lane traces one particle at a time; all state
// stays in registers.  A warp owns a 64-entry emission buffer in shared
// memory: when lanes run dry, the whole warp emits a batch of 32 new
// particles at once (step I, converged), then the dead lanes pop states from
// the buffer.  Lanes are therefore refilled as soon as their particle ends,
// whatever the spread of lifetimes, and emission never runs with a partial
// warp.  Particle ids come from a 64-bit global counter bumped once per
// batch.  Each flight k of particle pid draws its four uniforms from
// Philox4x32-10 at counter (k, 0, pid, instance), so the result does not
// depend on which lane or block traced the particle.
//
// Tallies.  Per particle the algebraic length along the flux axis is
// accumulated in the trajectory precision; per lane the sums over particles
// are kept as FP64 (FP64 runs) or compensated FP32 pairs (FP32 runs); each
// warp reduces them with shuffles before one FP64 atomic per quantity.
// Slab profiles (batch groups x bins, difference arrays for whole-bin runs)
// and the scattering-index split live in shared memory and are flushed once
// per block.  The transient grid takes int32 red-adds in global memory.
#pragma once

#include <stdint.h>

#include "device_math.cuh"
#include "le_mc_internal.h"

namespace lemc {

// Debug builds (-DLEMC_DEBUG) check the data-dependent indices of the trace
// kernels: an index out of its range sets FLAG_DEBUG_BOUNDS in the lane's
// status word and is replaced by 0, so the access stays in bounds and the
// run reports the defect instead of faulting.  Release builds compile the
// checks away.
#ifdef LEMC_DEBUG
#define LEMC_GUARD_INDEX(idx, n)                  \
    do {                                          \
        if (!((long long)(idx) >= 0 && (long long)(idx) < (long long)(n))) { \
            flags |= FLAG_DEBUG_BOUNDS;           \
            (idx) = 0;                            \
        }                                         \
    } while (0)
#define LEMC_DEBUG_CHECK(ok)                                 \
    do {                                                     \
        if (!(ok)) flags |= FLAG_DEBUG_BOUNDS;               \
    } while (0)
#else
#define LEMC_GUARD_INDEX(idx, n) \
    do {                         \
    } while (0)
#define LEMC_DEBUG_CHECK(ok) \
    do {                     \
    } while (0)
#endif

struct KernelArgs {
    TraceParams p;
    RoundKeys rk;
};

enum { HIT_NONE = 0, HIT_XLO = 1, HIT_XHI = 2, HIT_CYL = 3, HIT_YLO = 4, HIT_YHI = 5, HIT_ZLO = 6, HIT_ZHI = 7 };

constexpr int kBufSlots = 64;  // emission buffer entries per warp

// Fields of the emission buffer that a geometry or source may not need.
template <typename T, int N>
struct Slots {
    T v[N];
};
template <typename T>
struct Slots<T, 0> {};

// Emission buffer of one warp, structure of arrays.  y, z and the unit cell
// are kept only for POROUS geometries, the emission time only for PULSE, the
// batch instance only in batch mode.
template <typename R, bool YZ, bool TIME, bool INST>
struct alignas(16) EmitBuffer {
    R x[kBufSlots];
    R ox[kBufSlots], oy[kBufSlots], oz[kBufSlots];
    uint32_t pid[kBufSlots];
    uint32_t mode_sign[kBufSlots];  // mode | (sign < 0) << 31
    Slots<R, YZ ? kBufSlots : 0> y, z;
    Slots<uint32_t, YZ ? kBufSlots : 0> cell;  // cy | cz << 16
    Slots<R, TIME ? kBufSlots : 0> t;
    Slots<uint32_t, INST ? kBufSlots : 0> inst;
};

// Transient kernels defer the Eq. 3 samples of a segment: each lane leaves
// its segment's start point, direction, start time, speed, sign and first
// sample index here, and the whole warp then places the samples of all its
// lanes together at a point where every lane is converged (see flush_jobs in
// trace_kernel), so a lane whose segment spans many sample times no longer
// holds the other 31 lanes in a divergent loop.
template <typename R>
struct SampleJobs {
    R x[32], y[32], z[32], ox[32], oy[32], oz[32], t[32], v[32];
    int k0[32], sign[32], cell[32];  // cell: unit cell cy | cz << 16
};

// Steady-map kernels defer the map cells of a segment in the same way: each
// lane leaves, per map axis, the parameter of its segment's first cell-
// boundary crossing and the parameter step between crossings (the a-th
// crossing along y at ty0 + a dty; ty0 = +inf and dty = 0 for a segment
// parallel to the axis), its length, its time and z-flux weights per unit
// length, and one word packing its first map cell (j0, k0), its counts of
// map-cell boundaries crossed along y and z (nyc, nzc; each below the 64
// cells an axis may have), its batch group g (below 64) and the directions
// of travel along y and z (negative: bits 30, 31); the warp then adds the
// contributions of every crossed cell of every lane, one cell per lane.
template <typename R>
struct MapJobs {
    R ty0[32], dty[32], tz0[32], dtz[32], seg[32], wT[32], wQ[32];
    uint32_t pk[32];  // j0 | k0 << 6 | nyc << 12 | nzc << 18 | g << 24 | (sy < 0) << 30 | (sz < 0) << 31
};
static_assert(LE_MC_MAX_MAP <= 64 && LE_MC_MAX_BATCH <= 64, "map-job fields are packed in 6 bits each");

// The lane tallies of the steady FP32 pored-film kernel (its two compensated
// sums and seven counters, touched once per particle) live in shared memory,
// [kLaneWords][threads] words: the registers they free keep the segment's
// state out of local memory (60 bytes of spills per thread -> none, pored film
// 13.4 -> 13.0 ms for 2e7 particles).  For the film, which does not spill, the
// same measured 1.5 % slower; the transient and map kernels have no shared
// memory to spare for it.
constexpr int kLaneWords = 11;
template <typename R, int GEOM, int SRC, bool PROFILE, bool BATCH>
struct LaneTallyInSmem {
    static constexpr bool value =
        sizeof(R) == 4 && GEOM == LE_MC_GEOM_POROUS && SRC == LE_MC_SRC_GRADIENT && !PROFILE && !BATCH;
};

template <typename R, int GEOM, int SRC, bool BATCH = false>
using BufferOf = EmitBuffer<R, GEOM == LE_MC_GEOM_POROUS, SRC == LE_MC_SRC_PULSE, BATCH>;

// Compensated FP32 sum (Kahan: c carries the part of each addend that the
// running sum lost); plain sum for FP64.
template <typename R>
struct Acc {
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R v)
    {
        const R y = v - c;
        const R t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct Acc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename R>
__device__ __forceinline__ void load_props(const void* props, uint32_t mode, R& lam, R& vg)
{
    if constexpr (sizeof(R) == 4) {
        const float2 e = reinterpret_cast<const float2*>(props)[mode];
        lam = e.x;
        vg = e.y;
    } else {
        const double2 e = reinterpret_cast<const double2*>(props)[mode];
        lam = e.x;
        vg = e.y;
    }
}

// Problem constants in the trajectory precision (converted on the host).
template <typename R>
__device__ __forceinline__ const Consts<R>& consts_of(const TraceParams& P)
{
    if constexpr (sizeof(R) == 4) return P.c32;
    else return P.c64;
}

// What step I needs to know about the problem a particle belongs to: the
// run itself, or one instance of a batch (thickness, wall-source weights and
// signs, gradient direction factor), in the trajectory precision.
template <typename R>
struct EmitCtx {
    R L, wlo, whi, dir;
    int s_lo, s_hi;
    uint32_t inst;
};

template <typename R>
__device__ __forceinline__ EmitCtx<R> run_ctx(const TraceParams& P)
{
    const Consts<R>& K = consts_of<R>(P);
    EmitCtx<R> c;
    c.L = K.L;
    c.wlo = K.wlo;
    c.whi = K.whi;
    c.dir = K.grad_dir;
    c.s_lo = P.sign_lo;
    c.s_hi = P.sign_hi;
    c.inst = P.inst;
    return c;
}

template <typename R>
__device__ __forceinline__ EmitCtx<R> batch_ctx(const BatchInstance& b)
{
    EmitCtx<R> c;
    if constexpr (sizeof(R) == 4) {
        c.L = b.L32;
        c.wlo = b.wlo32;
        c.whi = b.whi32;
        c.dir = b.dir32;
    } else {
        c.L = b.L;
        c.wlo = fabs(b.dT_lo);
        c.whi = fabs(b.dT_hi);
        c.dir = b.dTdz > 0.0 ? -1.0 : 1.0;
    }
    c.s_lo = b.sign_lo;
    c.s_hi = b.sign_hi;
    c.inst = b.inst_id;
    return c;
}

// Batch instance holding global queue position p (offsets has n + 1 entries).
__device__ __forceinline__ uint32_t batch_find(const unsigned long long* offsets, uint32_t n, unsigned long long p)
{
    uint32_t lo = 0, hi = n;  // offsets[lo] <= p < offsets[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (offsets[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// Step I for one particle; returns false if a rejection loop ran out.  The
// emission alias table is read from global memory (once per particle, cached
// in L1), which leaves shared memory to the per-flight tables.
template <typename R, int GEOM, int SRC>
__device__ __forceinline__ bool emit_particle(const TraceParams& P, const EmitCtx<R>& E, const RoundKeys& rk,
                                              const uint2* alias_emit, uint32_t pid, R& x, R& y, R& z, R& ox,
                                              R& oy, R& oz, R& t, uint32_t& mode, int& sign, uint32_t& cy,
                                              uint32_t& cz)
{
    using M = DMath<R>;
    const Consts<R>& K = consts_of<R>(P);
    const uint4 r = philox4x32_10(make_uint4(0u, 0u, pid, E.inst), rk);
    mode = alias_draw(alias_emit, (uint32_t)P.n_modes, r.y);
    const R u0 = M::uniform(r.x), u2 = M::uniform(r.z), u3 = M::uniform(r.w);
    R sn, cs;
    M::sincos_2pi(u3, &sn, &cs);
    y = z = t = R(0);
    cy = cz = 0;
    bool ok = true;
    if constexpr (SRC == LE_MC_SRC_WALLS) {
        // isothermal walls: wall picked by |T_b - T_eq|, cosine law into the domain
        const bool lo = u0 * (E.wlo + E.whi) < E.wlo;
        const R mu = M::sqrt_(u2);
        const R st = M::sqrt_(fmax(R(0), R(1) - mu * mu));
        ox = lo ? mu : -mu;
        oy = st * cs;
        oz = st * sn;
        x = lo ? R(0) : E.L;
        sign = lo ? E.s_lo : E.s_hi;
    } else if constexpr (SRC == LE_MC_SRC_GRADIENT) {
        // Eq. 6: |cos| law about z, sign sgn(-cos dT/dz), even ids positive
        sign = (pid & 1u) ? -1 : 1;
        const R dir = (R)sign * E.dir;
        const R mu = dir * M::sqrt_(u2);
        const R st = M::sqrt_(fmax(R(0), R(1) - mu * mu));
        ox = st * cs;
        oy = st * sn;
        oz = mu;
        x = (GEOM == LE_MC_GEOM_BULK) ? R(0) : u0 * E.L;
        if constexpr (GEOM == LE_MC_GEOM_POROUS) {
            const R pitch = K.pitch, half = K.half, r2 = K.rad2;
            ok = false;
            for (uint32_t b = 1; b <= kMaxTries; ++b) {
                const uint4 q = philox4x32_10(make_uint4(0u, b, pid, E.inst), rk);
                const R Y = M::uniform(q.x) * pitch * (R)P.cells_y;
                const R Z = M::uniform(q.y) * pitch * (R)P.cells_z;
                int iy = (int)M::floor_(Y / pitch), iz = (int)M::floor_(Z / pitch);
                iy = min(max(iy, 0), P.cells_y - 1);
                iz = min(max(iz, 0), P.cells_z - 1);
                y = Y - (R)iy * pitch;
                z = Z - (R)iz * pitch;
                cy = (uint32_t)iy;
                cz = (uint32_t)iz;
                const R dy = y - half, dz = z - half;
                if (!(dy * dy + dz * dz < r2)) { ok = true; break; }
            }
        }
    } else if constexpr (SRC == LE_MC_SRC_INITIAL) {
        // initial condition: uniform in the heated layer (solid part), modes
        // weighted by C_b (table passed by the caller), isotropic, t = 0
        sign = P.init_sign;
        const R mu = R(2) * u2 - R(1);
        const R st = M::sqrt_(fmax(R(0), R(1) - mu * mu));
        ox = st * cs;
        oy = st * sn;
        oz = mu;
        x = K.init_lo + u0 * K.init_span;
        const R pitch = K.pitch, half = K.half, r2 = K.rad2;
        ok = false;
        for (uint32_t b = 1; b <= kMaxTries; ++b) {
            const uint4 q = philox4x32_10(make_uint4(0u, b, pid, E.inst), rk);
            const R Y = M::uniform(q.x) * pitch * (R)P.cells_y;
            const R Z = M::uniform(q.y) * pitch * (R)P.cells_z;
            int iy = (int)M::floor_(Y / pitch), iz = (int)M::floor_(Z / pitch);
            iy = min(max(iy, 0), P.cells_y - 1);
            iz = min(max(iz, 0), P.cells_z - 1);
            y = Y - (R)iy * pitch;
            z = Z - (R)iz * pitch;
            cy = (uint32_t)iy;
            cz = (uint32_t)iz;
            const R dy = y - half, dz = z - half;
            if (!(dy * dy + dz * dz < r2)) { ok = true; break; }
        }
    } else {  // PULSE on the top face x = L, all signs positive
        sign = 1;
        const R mu = M::sqrt_(u2);
        const R st = M::sqrt_(fmax(R(0), R(1) - mu * mu));
        ox = -mu;
        oy = st * cs;
        oz = st * sn;
        x = E.L;
        const R pitch = K.pitch, half = K.half, r2 = K.rad2;
        const R Dy = K.Dy, Dz = K.Dz;
        ok = false;
        for (uint32_t b = 1; b <= kMaxTries; ++b) {
            const uint4 q = philox4x32_10(make_uint4(0u, b, pid, E.inst), rk);
            const R rad = K.p_sx * M::sqrt_(R(2) * M::neg_log(M::uniform(q.x)));
            R s2, c2;
            M::sincos_2pi(M::uniform(q.y), &s2, &c2);
            R Y = K.p_y0 + rad * c2;
            R Z = K.p_z0 + rad * s2;
            Y -= Dy * M::floor_(Y / Dy);
            Z -= Dz * M::floor_(Z / Dz);
            int iy = (int)M::floor_(Y / pitch), iz = (int)M::floor_(Z / pitch);
            iy = min(max(iy, 0), P.cells_y - 1);
            iz = min(max(iz, 0), P.cells_z - 1);
            y = Y - (R)iy * pitch;
            z = Z - (R)iz * pitch;
            cy = (uint32_t)iy;
            cz = (uint32_t)iz;
            const R dy = y - half, dz = z - half;
            if (!(dy * dy + dz * dz < r2)) { ok = true; break; }
        }
        t = K.p_tc;
        bool tok = false;
        for (uint32_t b = kTimeBlock0; b < kTimeBlock0 + kMaxTries; ++b) {
            const uint4 q = philox4x32_10(make_uint4(0u, b, pid, E.inst), rk);
            R s2, c2;
            M::sincos_2pi(M::uniform(q.y), &s2, &c2);
            const R t0 = K.p_tc + K.p_st * M::sqrt_(R(2) * M::neg_log(M::uniform(q.x))) * c2;
            if (t0 >= R(0)) { t = t0; tok = true; break; }
        }
        ok = ok && tok;
    }
    return ok;
}

constexpr float kLn2f = 0.693147180559945f;

template <typename R, int SRC, bool PROFILE>
struct FusedTable {
    static constexpr bool value = sizeof(R) == 4 && SRC != LE_MC_SRC_PULSE && SRC != LE_MC_SRC_INITIAL && !PROFILE;
};

// Bytes of the per-mode tables at the start of shared memory (16-aligned).
template <typename R, int SRC, bool PROFILE>
__host__ __device__ inline size_t table_bytes(int n_modes)
{
    const size_t per_mode = FusedTable<R, SRC, PROFILE>::value ? 16 : (2 * sizeof(R) + 8);
    return ((size_t)n_modes * per_mode + 15) & ~(size_t)15;
}

// DIFF: every wall (both planes, and the pores) is diffuse, relaxation
// events are isotropic (the paper's base case) and no flux split by
// scattering index is asked for, so the wall law needs no per-wall lookup
// and no specular, absorbing or partial branch, the direction law no
// anisotropic branch, and the loop no H_j bookkeeping (which cost 9 % of the
// film kernel's time).
template <typename R, int GEOM, int SRC, bool PROFILE, bool BATCH, bool DIFF>
__device__ __forceinline__ void trace_body(const KernelArgs& args)
{
    using M = DMath<R>;
    using Buf = BufferOf<R, GEOM, SRC, BATCH>;
    static_assert(sizeof(Buf) >= 32 * sizeof(uint4) && sizeof(Buf) % 16 == 0,
                  "assisted rounds keep 32 random words in a warp's emission buffer");
    constexpr bool POROUS = (GEOM == LE_MC_GEOM_POROUS);
    constexpr bool TRANSIENT = (SRC == LE_MC_SRC_PULSE || SRC == LE_MC_SRC_INITIAL);
    constexpr bool AXIS_X = (SRC == LE_MC_SRC_WALLS);
    // the flux split by scattering index (a steady estimator): not in DIFF
    // kernels (runs that ask for it use the general kernel) nor transient ones
    constexpr bool HJ = !DIFF && !TRANSIENT;
    // Kernels whose estimators never need the group velocity (steady path
    // integrals) keep one 16-byte word per mode: (threshold, alias,
    // Lambda_j, Lambda_alias), so an Eq. 2 redraw is a single shared load.
    constexpr bool FUSED = FusedTable<R, SRC, PROFILE>::value;
    const TraceParams& P = args.p;
    const RoundKeys& rk = args.rk;
    // the per-warp queue claims and emission buffers assume whole warps and
    // at most 512 threads; the host validates launch shapes, and a kernel
    // given any other reports it and traces nothing
    if ((blockDim.x & 31u) != 0u || blockDim.x > 512u) {
        if (threadIdx.x == 0) atomicOr(P.flags, FLAG_BAD_LAUNCH);
        return;
    }

    extern __shared__ __align__(16) unsigned char smem[];
    const int n_modes = P.n_modes;
    R* s_props = reinterpret_cast<R*>(smem);
    uint2* s_scat = reinterpret_cast<uint2*>(smem + (size_t)n_modes * 2 * sizeof(R));
    uint4* s_fused = reinterpret_cast<uint4*>(smem);
    size_t off = table_bytes<R, SRC, PROFILE>(n_modes);
    Buf* s_buf = reinterpret_cast<Buf*>(smem + off);
    const int n_warps = blockDim.x >> 5;
    off += (size_t)n_warps * sizeof(Buf);
    SampleJobs<R>* s_jobs = reinterpret_cast<SampleJobs<R>*>(smem + off);
    if constexpr (TRANSIENT) off += (size_t)n_warps * sizeof(SampleJobs<R>);
    MapJobs<R>* s_mjobs = reinterpret_cast<MapJobs<R>*>(smem + off);
    if constexpr (PROFILE && POROUS) off += (size_t)n_warps * sizeof(MapJobs<R>);
    // FP32 copy of this block's slab profile or steady maps (drained into
    // the FP64 sums), when the host found room for it
    constexpr bool PROF32 = PROFILE && sizeof(R) == 4;
    float* s_prof32 = reinterpret_cast<float*>(smem + off);
    const int prof32_len = (PROF32 && P.prof_smem)
                               ? (POROUS ? 2 * P.n_batch * P.map_ny * P.map_nz : 4 * P.n_batch * (P.n_bins_x + 1))
                               : 0;
    off += (size_t)prof32_len * sizeof(float);
    off = (off + 7) & ~(size_t)7;
    // batch mode: per-instance sums [n][2] and counters [n][CNT_N] of this block
    const bool inst_in_smem = BATCH && P.n_instances <= kBatchSmemMax;
    const int inst_len = inst_in_smem ? P.n_instances : 0;
    double* s_isum = reinterpret_cast<double*>(smem + off);
    unsigned long long* s_icnt = reinterpret_cast<unsigned long long*>(smem + off + (size_t)inst_len * 2 * sizeof(double));
    off += (size_t)inst_len * (2 * sizeof(double) + CNT_N * sizeof(unsigned long long));
    constexpr bool LANE_SMEM = LaneTallyInSmem<R, GEOM, SRC, PROFILE, BATCH>::value;
    // (LANE_SMEM) this thread's lane tallies: word k at lt[k * blockDim.x]
    uint32_t* const lt = reinterpret_cast<uint32_t*>(smem + off) + threadIdx.x;
    const int lts = (int)blockDim.x;

    // mode tables and block tallies
    for (int i = threadIdx.x; i < n_modes; i += blockDim.x) {
        R lam, vg;
        load_props<R>(P.props, (uint32_t)i, lam, vg);
        const uint2 e = P.alias_scat[i];
        if constexpr (FUSED) {
            // (Lambda ln 2: the flight -Lambda ln u is then -(Lambda ln 2) log2 u)
            R lam_a, vg_a;
            load_props<R>(P.props, e.y, lam_a, vg_a);
            s_fused[i] = make_uint4(e.x, e.y, __float_as_uint((float)lam * kLn2f),
                                    __float_as_uint((float)lam_a * kLn2f));
        } else {
            s_props[2 * i] = lam;
            s_props[2 * i + 1] = vg;
            s_scat[i] = e;
        }
    }
    for (int i = threadIdx.x; i < prof32_len; i += blockDim.x) s_prof32[i] = 0.0f;
    for (int i = threadIdx.x; i < 2 * inst_len; i += blockDim.x) s_isum[i] = 0.0;
    for (int i = threadIdx.x; i < CNT_N * inst_len; i += blockDim.x) s_icnt[i] = 0ull;
    if constexpr (LANE_SMEM)
        for (int k = 0; k < kLaneWords; ++k) lt[k * lts] = 0u;
    __syncthreads();

    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    Buf& buf = s_buf[threadIdx.x >> 5];
    // queue positions: the long-first list, then positions 0 .. n_pos - 1
    // (particle ids of the run, or the concatenated instances of a batch)
    // minus those already listed
    const unsigned long long n_pos = BATCH ? P.offsets[P.n_instances] : (unsigned long long)P.n_particles;
    // The extreme list is used all or nothing: if classification found more
    // extreme particles than it holds, which ones fit depended on the order
    // of atomics, so none is traced apart and the (full, contiguous) extreme
    // region joins the long-first list instead.
    const uint32_t raw_ext = (P.long_list && P.ext_cap > 0) ? P.long_count[1] : 0u;
    const bool ext_overflow = raw_ext > P.ext_cap;
    const uint32_t n_ext = ext_overflow ? 0u : raw_ext;
    const uint32_t n_long0 = P.long_list ? min(P.long_count[0], P.long_cap) : 0u;
    const uint32_t n_long = ext_overflow ? P.ext_cap + n_long0 : n_long0;
    const uint32_t* long_region = P.long_list ? (ext_overflow ? P.long_list : P.long_list + P.ext_cap) : nullptr;
    const unsigned long long q_total = (unsigned long long)n_long + n_pos;
    const int refill_min = P.refill_min > 1 ? P.refill_min : 1;
    const Consts<R>& K = consts_of<R>(P);
    const R L = K.L;
    const R pitch = K.pitch, half = K.half, rad = K.rad, rad2 = K.rad2;
    const R big = M::big();
    // slab-profile bin width and bins per unit length (kernel-uniform; a bin
    // index is floor(x / dx), formed as a product)
    const R prof_dx = (PROFILE && !POROUS && P.n_bins_x > 0) ? L / (R)P.n_bins_x : R(1);
    const R prof_ib = (PROFILE && !POROUS && P.n_bins_x > 0) ? (R)P.n_bins_x / L : R(1);
    // anisotropic relaxation-event direction law (kernel-uniform)
    const bool aniso = !DIFF && P.aniso != 0;
    const R hg = K.g;
    // collision cap (first free path): needs its own check only where periodic
    // faces end segments too; elsewhere the host folds it into max_events
    const bool col_cap = POROUS && P.max_collisions > 0u;
    // partially specular walls present (kernel-uniform)
    const bool any_partial = !DIFF && (P.wall_lo == LE_MC_WALL_PARTIAL || P.wall_hi == LE_MC_WALL_PARTIAL ||
                                       (POROUS && P.pore_wall == LE_MC_WALL_PARTIAL));

    // particle state
    R x = 0, y = 0, z = 0, ox = 0, oy = 0, oz = 1, t = 0, lam = 1, vg = 1;
    R Lacc = 0, hrun = 0, x0 = 0, t0 = 0;
    uint32_t pid = 0, n_seg = 0, n_scat = 0, n_wall = 0, n_per = 0, mode0 = 0;
    int pgroup = 0;  // batch group of the particle (profiles and maps), set once per particle
    PhiloxLane plane = {0u, 0u, 0u};  // per-particle part of the flights' random words
    int cy = 0, cz = 0, sign = 1, fate = FATE_MAX_EVENTS;
    bool alive = false, pending = false;
    // problem of the current particle (batch mode: its instance)
    uint32_t bidx = 0, instw = P.inst;
    R Lp = L;

    // lane accumulators
    Acc<R> acc_sL, acc_sL2;
    uint32_t c_part = 0, c_seg = 0, c_scat = 0, c_wall = 0, c_per = 0, c_trunc = 0, c_abs = 0;
    uint32_t flags = 0;

    // FP64 tally reduction into global memory: the add is done by the L2's
    // atomic units, and FP32 kernels widen the value on the integer units, so
    // no tally arithmetic reaches the (narrow) FP64 pipe of the SM
    auto red64 = [&](double* dst, R v) {
        const double d = M::to_f64(v);
#ifdef LEMC_DEBUG
        if (!(d == (double)v) && v == v) flags |= FLAG_DEBUG_BOUNDS;
#endif
        atomicAdd(dst, d);
    };

    // Slab profile or map entry i: into this block's FP32 copy (a shared-
    // memory add, which the hardware carries out as a compare-and-swap loop)
    // when it has one, else straight into the FP64 sums.  Each warp drains
    // its share of the copy (atomic exchange with 0, then one FP64 reduction
    // per nonzero entry) every kProfDrainEvery loop iterations, so an FP32
    // partial sum holds only the few dozen contributions made to its entry in
    // between; the block drains everything at the end.
    auto prof_add = [&](size_t i, R v) {
        if (PROF32 && prof32_len > 0) atomicAdd(&s_prof32[i], (float)v);
        else red64(P.prof + i, v);
    };
    int drain_it = 0;
    auto drain_prof = [&](int first, int end) {
        for (int i = first + lane; i < end; i += 32) {
            const float v = atomicExch(&s_prof32[i], 0.0f);
            if (v != 0.0f) red64(P.prof + i, (R)v);
        }
    };

    int cnt = 0;         // emission buffer fill (warp-uniform)
    bool qdone = false;  // particle queue exhausted (warp-uniform)
    // queue positions this warp has claimed but not yet emitted (warp-uniform);
    // claims are `chunk` positions at a time, except inside the long-first
    // list: there a claim is 32 positions, one particle per lane, because
    // each listed particle can run for as long as a lane's whole share of the
    // ordinary ones, and a larger claim would queue several of them behind
    // one another on one lane (claims much smaller than a warp spread them
    // over every warp instead, which leaves a few busy lanes per warp at the
    // end: measured slower on the film)
    const unsigned long long chunk = P.chunk >= 32 ? (unsigned long long)P.chunk : 32ull;
    const unsigned long long long_claim = 32ull;
    unsigned long long w_next = 0, w_end = 0;
    uint32_t cur_b = 0xFFFFFFFFu;  // batch instance the lane accumulators belong to

    // batch mode: move the lane accumulators to instance b's totals
    auto flush_lane = [&](uint32_t b) {
        if (b == 0xFFFFFFFFu) return;
        const double v[2] = {acc_sL.value(), acc_sL2.value()};
        const uint32_t c[CNT_N] = {c_part, c_seg, c_scat, c_wall, c_per, c_trunc, c_abs};
        if (inst_in_smem) {
            atomicAdd(&s_isum[2 * b], v[0]);
            atomicAdd(&s_isum[2 * b + 1], v[1]);
            for (int i = 0; i < CNT_N; ++i)
                if (c[i]) atomicAdd(&s_icnt[CNT_N * b + i], (unsigned long long)c[i]);
        } else {
            atomicAdd(&P.inst_sums[2 * b], v[0]);
            atomicAdd(&P.inst_sums[2 * b + 1], v[1]);
            for (int i = 0; i < CNT_N; ++i)
                if (c[i]) atomicAdd(&P.inst_counters[(size_t)CNT_N * b + i], (unsigned long long)c[i]);
        }
        acc_sL = Acc<R>();
        acc_sL2 = Acc<R>();
        c_part = c_seg = c_scat = c_wall = c_per = c_trunc = c_abs = 0;
    };

    // Eq. 3 tally of one sample: the particle's cell at t'_k adds its sign.
    // (FP32: products with host-computed reciprocals; FP64: the divisions
    // exactly as the oracle forms them.)
    auto place_sample = [&](int k, R x0, R y0, R z0, R dx, R dy, R dz, R t0, R v, int s, int ccy, int ccz) {
        const R d = v * (((R)k + R(0.5)) * K.sample_dt - t0);
        const R px = x0 + dx * d, py = (R)ccy * pitch + (y0 + dy * d), pz = (R)ccz * pitch + (z0 + dz * d);
        int ix, iy, iz;
        if constexpr (sizeof(R) == 4) {
            ix = (int)M::floor_(px * K.gsx);
            iy = (int)M::floor_(py * K.gsy);
            iz = (int)M::floor_(pz * K.gsz);
        } else {
            ix = (int)M::floor_(px / L * (R)P.gx);
            iy = (int)M::floor_(py / K.Dy * (R)P.gy);
            iz = (int)M::floor_(pz / K.Dz * (R)P.gz);
        }
        // (a sample on the domain's far faces rounds one cell out; anything
        // further means the position left the domain)
        LEMC_DEBUG_CHECK(ix >= -1 && ix <= P.gx && iy >= -1 && iy <= P.gy && iz >= -1 && iz <= P.gz);
        ix = min(max(ix, 0), P.gx - 1);
        iy = min(max(iy, 0), P.gy - 1);
        iz = min(max(iz, 0), P.gz - 1);
        const size_t cell = (((size_t)k * P.gz + iz) * P.gy + iy) * P.gx + ix;
        atomicAdd(&P.grid[cell], s);
    };
    // Place every deferred sample of the warp (all 32 lanes converged): item j
    // of the warp's total belongs to the first lane whose inclusive prefix
    // count exceeds j (binary search over the lanes by shuffles).
    int job_n = 0;
    auto flush_jobs = [&]() {
        const int total = __reduce_add_sync(FULL, (unsigned)job_n);
        if (total == 0) return;
        int inc = job_n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += v;
        }
        const int excl = inc - job_n;
        const SampleJobs<R>& J = s_jobs[threadIdx.x >> 5];
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int j = base + lane;
            int own = 0;
#pragma unroll
            for (int bit = 16; bit > 0; bit >>= 1) {
                const int v = __shfl_sync(FULL, inc, own + bit - 1);
                if (v <= j) own += bit;
            }
            LEMC_GUARD_INDEX(own, 32);
            const int own_excl = __shfl_sync(FULL, excl, own);
            if (j < total)
                place_sample(J.k0[own] + (j - own_excl), J.x[own], J.y[own], J.z[own], J.ox[own], J.oy[own], J.oz[own],
                             J.t[own], J.v[own], J.sign[own], J.cell[own] & 0xFFFF, J.cell[own] >> 16);
        }
        __syncwarp();
        job_n = 0;
    };

    // Map-cell boundaries crossed by a segment of length seg that starts at
    // coordinate u (within the unit cell) in map cell c0 of n, with direction
    // component o and r = 1 / o (0: parallel): crossing a (a = 0, 1, ...),
    // at coordinate (c0 + s a + [s > 0]) h (s the direction's sign), is
    // reached at parameter t(a) = t0 + a dt, with t0 = ((c0 + [s > 0]) h -
    // u) r and dt = h |r|; a boundary counts when t(a) < seg and the next
    // cell is on the map.  The estimate from the end point is corrected by
    // the comparisons (at most one step each way).
    auto map_crossings = [&](R u, R o, R r, R t0, R dt, R seg, int c0, int n, R ih) -> int {
        if (r == R(0)) return 0;
        const int sg = r > R(0) ? 1 : -1;
        const int amax = sg > 0 ? n - 1 - c0 : c0;
        auto t_of = [&](int a) { return t0 + (R)a * dt; };  // as the walk evaluates them
        const R ue = u + o * seg;
        const int ce = min(max((int)M::floor_(ue * ih), 0), n - 1);
        int m = min(max(sg > 0 ? ce - c0 : c0 - ce, 0), amax);
        while (m > 0 && !(t_of(m - 1) < seg)) --m;
        while (m < amax && t_of(m) < seg) ++m;
        return m;
    };
    // Cell i (0 .. nyc + nzc) of a segment's walk over the map: after a
    // crossings along y and b = i - a along z, a being the number of y
    // crossings among the first i in order of parameter (y first on ties),
    // found by a merge-path binary search; the segment spends the parameter
    // interval [latest crossing so far, earliest next crossing or seg] in
    // it, and adds d wT and d wQ to the cell's sums of batch group g.
    auto map_item = [&](R ty0, R dty, R tz0, R dtz, R seg, R wT, R wQ, uint32_t pk, int i) {
        const int j0 = (int)(pk & 63u), k0 = (int)((pk >> 6) & 63u);
        const int nyc = (int)((pk >> 12) & 63u), nzc = (int)((pk >> 18) & 63u), g = (int)((pk >> 24) & 63u);
        const int sy = (pk >> 30) & 1u ? -1 : 1, sz = (pk >> 31) ? -1 : 1;
        auto ty = [&](int a) { return ty0 + (R)a * dty; };
        auto tz = [&](int b) { return tz0 + (R)b * dtz; };
        int lo = max(0, i - nzc), hi = min(i, nyc);
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const R tzm = (i - mid < nzc) ? tz(i - mid) : big;
            if (ty(mid - 1) <= tzm) lo = mid;
            else hi = mid - 1;
        }
        const int a = lo, b = i - lo;
        const R t_in = fmax(a > 0 ? ty(a - 1) : R(0), b > 0 ? tz(b - 1) : R(0));
        const R t_out = fmin(fmin(ty(a), tz(b)), seg);
        const R d = t_out - t_in;
        if (d > R(0)) {
            // (entries of [2][n_batch][map_nz][map_ny]: below 2^19)
            const int ny = P.map_ny, cells = ny * P.map_nz;
            int c = (k0 + sz * b) * ny + (j0 + sy * a);
            LEMC_GUARD_INDEX(c, cells);
            prof_add((size_t)(g * cells + c), d * wT);
            prof_add((size_t)((P.n_batch + g) * cells + c), d * wQ);
        }
    };
    // Add every deferred map cell of the warp (all 32 lanes converged): item
    // j of the warp's total belongs to the first lane whose inclusive prefix
    // count exceeds j, as for the sample jobs.
    int mjob_n = 0;
    auto flush_map_jobs = [&]() {
        const int total = __reduce_add_sync(FULL, (unsigned)mjob_n);
        if (total == 0) return;
        int inc = mjob_n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += v;
        }
        const int excl = inc - mjob_n;
        const MapJobs<R>& J = s_mjobs[threadIdx.x >> 5];
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int j = base + lane;
            int own = 0;
#pragma unroll
            for (int bit = 16; bit > 0; bit >>= 1) {
                const int v = __shfl_sync(FULL, inc, own + bit - 1);
                if (v <= j) own += bit;
            }
            LEMC_GUARD_INDEX(own, 32);
            const int own_excl = __shfl_sync(FULL, excl, own);
            if (j < total)
                map_item(J.ty0[own], J.dty[own], J.tz0[own], J.dtz[own], J.seg[own], J.wT[own], J.wQ[own], J.pk[own],
                         j - own_excl);
        }
        __syncwarp();
        mjob_n = 0;
    };

    // ---- one segment: steps II-VI, from the segment's four random words r
    // (counter (n_seg + 1, 0, pid, instance): known before the segment runs)
    auto segment = [&](const uint4 r, const bool coop) {
        // step II: flight to the next relaxation event (as a length)
        R ell;
        if constexpr (FUSED) ell = -(lam * __log2f(M::uniform(r.x)));  // lam holds Lambda ln 2 here
        else ell = lam * M::neg_log(M::uniform(r.x));
        // step III: first boundary along the ray
        R d_b = big;
        int kind = HIT_NONE;
        R wpos = R(0);  // position of the x wall ahead
        if constexpr (GEOM != LE_MC_GEOM_BULK) {
            // distance to the wall ahead; a flight parallel to the walls gets
            // an infinite (or NaN, never <= ell) distance and no hit
            const bool up = ox > R(0);
            wpos = up ? Lp : R(0);
            d_b = M::div(fabs(wpos - x), fabs(ox));
            kind = up ? HIT_XHI : HIT_XLO;
        }
        if constexpr (POROUS) {
            if (rad > R(0)) {
                const R ry = y - half, rz = z - half;
                const R a = oy * oy + oz * oz;
                const R b = ry * oy + rz * oz;
                const R c = ry * ry + rz * rz - rad2;
                if (a > R(0) && b < R(0)) {
                    const R disc = b * b - a * c;
                    if (disc >= R(0)) {
                        R tc = M::div(c, M::sqrt_(disc) - b);
                        tc = fmax(tc, R(0));
                        if (tc < d_b) { d_b = tc; kind = HIT_CYL; }
                    }
                }
            }
            // unit-cell faces ahead in y and z, one division each (a flight
            // parallel to a face pair gets an infinite or NaN distance there)
            const R tfy = M::div(oy > R(0) ? pitch - y : y, fabs(oy));
            if (tfy < d_b) { d_b = tfy; kind = oy > R(0) ? HIT_YHI : HIT_YLO; }
            const R tfz = M::div(oz > R(0) ? pitch - z : z, fabs(oz));
            if (tfz < d_b) { d_b = tfz; kind = oz > R(0) ? HIT_ZHI : HIT_ZLO; }
        }
        bool hit = (kind != HIT_NONE) && (d_b <= ell);
        if constexpr (sizeof(R) == 4 && SRC == LE_MC_SRC_WALLS && GEOM == LE_MC_GEOM_PLANES) {
            // Absorbing walls decide a particle's fate: when the FP32 flight
            // and wall distances are within a few ulp of each other (grazing
            // flights make the wall distance large and its rounding
            // relatively coarse), redo the comparison in FP64 from the same
            // inputs.
            const int wtype = (kind == HIT_XLO) ? P.wall_lo : P.wall_hi;
            if (wtype == LE_MC_WALL_BLACK && fabsf(d_b - ell) <= 8.0f * 1.1920929e-7f * fmaxf(d_b, ell)) {
                const double u = (double)M::uniform(r.x);
                // (a fused table holds Lambda ln 2, the flight is then -(Lambda ln 2) log2 u)
                const double ell64 = FUSED ? (double)lam * -log2(u) : (double)lam * -log(u);
                const double d64 = ((ox > 0.0f) ? ((double)Lp - (double)x) : (double)x) / fabs((double)ox);
                hit = d64 <= ell64;
            }
        }
        R seg = hit ? d_b : ell;
        if constexpr (sizeof(R) == 4 && SRC == LE_MC_SRC_WALLS && GEOM == LE_MC_GEOM_PLANES) {
            seg = hit ? d_b : fminf(ell, d_b);  // a relaxation decided in FP64 happens on this side of the wall
        }
        R x_new = x + ox * seg;
        if (hit && (kind == HIT_XLO || kind == HIT_XHI)) x_new = wpos;

        // end time of the segment, computed once: the sample windows [t, t_b)
        // of consecutive segments must tile time exactly (no sample lost or
        // counted twice), so the particle's next start is this same value
        R t_b = t;
        if constexpr (TRANSIENT) t_b = t + seg / vg;
        // step V: contribution of the segment
        if constexpr (TRANSIENT) {
            // Eq. 3: the sample times t'_k in [t, t_b), up to t_final: a
            // contiguous index range [k_lo, k_end), found exactly from
            // rounded estimates with the same comparisons a scan would make
            const R dts = K.sample_dt;
            const R t_end = fmin(t_b, K.t_final);
            const int ns = P.n_samples;
            auto ts_of = [&](int k) { return ((R)k + R(0.5)) * dts; };
            int k_lo, k_end;
            if constexpr (sizeof(R) == 4) {
                k_lo = (int)ceil(t * K.inv_dt - R(0.5)) - 1;
                k_end = (int)ceil(t_end * K.inv_dt - R(0.5)) - 1;
            } else {
                k_lo = (int)ceil(t / dts - R(0.5)) - 1;
                k_end = (int)ceil(t_end / dts - R(0.5)) - 1;
            }
            // Both start one below the true bound (the rounded quotient errs by
            // less than one sample for n_samples <= 2^20, which the host
            // enforces) and are clamped into [0, n_samples]: a segment after
            // the last sample time has none, however far t_final lies beyond.
            k_lo = min(max(k_lo, 0), ns);
            while (k_lo < ns && ts_of(k_lo) < t) ++k_lo;
            k_end = min(max(k_end, k_lo), ns);
            while (k_end < ns && ts_of(k_end) < t_b && ts_of(k_end) <= t_end) ++k_end;
            const int n_s = k_end - k_lo;
            // (cy, cz are kept wrapped into the periodic domain)
            if (coop) {
                job_n = n_s;
                if (n_s > 0) {
                    SampleJobs<R>& J = s_jobs[threadIdx.x >> 5];
                    J.x[lane] = x;
                    J.y[lane] = y;
                    J.z[lane] = z;
                    J.cell[lane] = cy | (cz << 16);
                    J.ox[lane] = ox;
                    J.oy[lane] = oy;
                    J.oz[lane] = oz;
                    J.t[lane] = t;
                    J.v[lane] = vg;
                    J.k0[lane] = k_lo;
                    J.sign[lane] = sign;
                }
            } else {
                for (int k = k_lo; k < k_end; ++k) place_sample(k, x, y, z, ox, oy, oz, t, vg, sign, cy, cz);
            }
        }
        if constexpr (PROFILE && POROUS) {
            // steady maps (Eq. 4 per map cell): the segment adds s x (time
            // over the cell) and s x (z displacement over the cell) to every
            // cell of the (y, z) map that it crosses.  Here only the cell
            // range is found: the first cell, and how many cell boundaries
            // the segment crosses along y and along z before it ends (the
            // a-th crossing's parameter is formed directly as t0 + a dt, one
            // rounding, so nothing drifts, and counted with the same values
            // the walk uses); the cells are added by map_item, converged across
            // the warp (flush_map_jobs) or, in the assisted rounds, by this
            // lane alone.
            const int ny = P.map_ny, nz = P.map_nz;
            // (a position on the cell's far faces rounds at most one map cell out)
            LEMC_DEBUG_CHECK(y * K.map_iy > R(-1) && y * K.map_iy < (R)(ny + 1) && z * K.map_iz > R(-1) &&
                             z * K.map_iz < (R)(nz + 1));
            const int j0 = min(max((int)M::floor_(y * K.map_iy), 0), ny - 1);
            const int k0 = min(max((int)M::floor_(z * K.map_iz), 0), nz - 1);
            const R ry = oy != R(0) ? M::div(R(1), oy) : R(0);
            const R rz = oz != R(0) ? M::div(R(1), oz) : R(0);
            // crossing parameters: the a-th y boundary crossed lies at
            // (j0 + sy a + uy) dy, reached at ty0 + a dty
            const R ty0 = ry != R(0) ? ((R)(j0 + (ry > R(0) ? 1 : 0)) * K.map_dy - y) * ry : big;
            const R dty = ry != R(0) ? K.map_dy * fabs(ry) : R(0);
            const R tz0 = rz != R(0) ? ((R)(k0 + (rz > R(0) ? 1 : 0)) * K.map_dz - z) * rz : big;
            const R dtz = rz != R(0) ? K.map_dz * fabs(rz) : R(0);
            const int nyc = map_crossings(y, oy, ry, ty0, dty, seg, j0, ny, K.map_iy);
            const int nzc = map_crossings(z, oz, rz, tz0, dtz, seg, k0, nz, K.map_iz);
            const int g = pgroup;
            const R wT = M::div((R)sign, vg), wQ = (R)sign * oz;
            const uint32_t pk = (uint32_t)j0 | ((uint32_t)k0 << 6) | ((uint32_t)nyc << 12) | ((uint32_t)nzc << 18) |
                                ((uint32_t)g << 24) | (ry < R(0) ? (1u << 30) : 0u) | (rz < R(0) ? (1u << 31) : 0u);
            if (coop) {
                mjob_n = 1 + nyc + nzc;
                MapJobs<R>& J = s_mjobs[threadIdx.x >> 5];
                J.ty0[lane] = ty0;
                J.dty[lane] = dty;
                J.tz0[lane] = tz0;
                J.dtz[lane] = dtz;
                J.seg[lane] = seg;
                J.wT[lane] = wT;
                J.wQ[lane] = wQ;
                J.pk[lane] = pk;
            } else {
                for (int i = 0; i <= nyc + nzc; ++i) map_item(ty0, dty, tz0, dtz, seg, wT, wQ, pk, i);
            }
        }
        if constexpr (PROFILE && !POROUS) {
            // time spent in each bin along x, and the displacement along the
            // flux axis made there: x for the walls source (slab), z for the
            // gradient source (the in-plane flux of a film by depth); arrays
            // [4][n_batch][n_bins_x + 1] (T direct, T difference, q direct, q
            // difference) of FP64 sums, through prof_add
            const int nb = P.n_bins_x;
            const R dx = prof_dx;
            const int g = pgroup;
            const size_t stride = (size_t)nb + 1;
            const size_t Td = (0 * (size_t)P.n_batch + g) * stride;
            const size_t Tr = (1 * (size_t)P.n_batch + g) * stride;
            const size_t qd = (2 * (size_t)P.n_batch + g) * stride;
            const size_t qr = (3 * (size_t)P.n_batch + g) * stride;
            const R lo = fmin(x, x_new), hi = fmax(x, x_new);
            int k0 = (int)M::floor_(lo * prof_ib), k1 = (int)M::floor_(hi * prof_ib);
            // (a wall position rounds at most one bin out)
            LEMC_DEBUG_CHECK(k0 >= -1 && k1 <= nb);
            k0 = min(max(k0, 0), nb - 1);
            k1 = min(max(k1, 0), nb - 1);
            // signed contributions: in FP64 kernels a product by +-1 is a
            // flip of the sign bit on the integer units (the FP64 pipe is
            // narrow), bit for bit the same value
            auto sgn = [&](R v, int s) -> R {
                if constexpr (sizeof(R) == 8)
                    return __longlong_as_double(__double_as_longlong(v) ^ (s < 0 ? (long long)(1ull << 63) : 0ll));
                else
                    return (R)s * v;
            };
            if (ox == R(0)) {
                prof_add(Td + k0, sgn(seg / vg, sign));
                if constexpr (!AXIS_X) prof_add(qd + k0, sgn(oz * seg, sign));
            } else {
                const R w = R(1) / (vg * fabs(ox));  // time per unit x
                // displacement along the flux axis per unit x: +-1 for the
                // walls source (x itself), oz / |ox| for the gradient source
                const R qs = AXIS_X ? R(1) : M::div(oz, fabs(ox));
                const int sq = AXIS_X ? (ox > R(0) ? sign : -sign) : sign;
                if (k0 == k1) {
                    const R len = hi - lo;
                    prof_add(Td + k0, sgn(len * w, sign));
                    prof_add(qd + k0, sgn(AXIS_X ? len : len * qs, sq));
                } else {
                    const R la = (R)(k0 + 1) * dx - lo;  // partial first bin
                    const R lb = hi - (R)k1 * dx;        // partial last bin
                    prof_add(Td + k0, sgn(la * w, sign));
                    prof_add(qd + k0, sgn(AXIS_X ? la : la * qs, sq));
                    prof_add(Td + k1, sgn(lb * w, sign));
                    prof_add(qd + k1, sgn(AXIS_X ? lb : lb * qs, sq));
                    if (k1 > k0 + 1) {  // whole bins k0+1 .. k1-1
                        const R tw = dx * w, qw = AXIS_X ? dx : dx * qs;
                        prof_add(Tr + k0 + 1, sgn(tw, sign));
                        prof_add(Tr + k1, sgn(tw, -sign));
                        prof_add(qr + k0 + 1, sgn(qw, sq));
                        prof_add(qr + k1, sgn(qw, -sq));
                    }
                }
            }
        }
        const R dL = AXIS_X ? (x_new - x) : oz * seg;
        Lacc += dL;
        if constexpr (HJ) hrun += dL;

        // steps IVa / IVb.  Every lane evaluates the same straight-line code
        // and keeps its own outcome through selects, so walls and relaxation
        // events do not split the warp.
        x = x_new;
        if constexpr (POROUS) {
            y += oy * seg;
            z += oz * seg;
        }
        if constexpr (TRANSIENT) t = t_b;
        ++n_seg;
        const bool scat = !hit;
        int wall = -1;
        if constexpr (DIFF && !POROUS) {
            // (every boundary of a film is a diffuse wall: folded below)
        } else if constexpr (DIFF) {
            wall = (hit && kind <= HIT_CYL) ? (int)LE_MC_WALL_DIFFUSE : -1;
        } else if constexpr (GEOM != LE_MC_GEOM_BULK) {
            wall = (kind == HIT_XLO) ? P.wall_lo : ((kind == HIT_XHI) ? P.wall_hi : -1);
            if constexpr (POROUS) wall = (kind == HIT_CYL) ? P.pore_wall : wall;
            wall = hit ? wall : -1;
            // partially specular wall: specular with probability p, decided by
            // the flight's second uniform (a relaxation's mode draw otherwise)
            if (any_partial && wall == LE_MC_WALL_PARTIAL) {
                const R p = (kind == HIT_XLO) ? K.spec_lo : ((kind == HIT_XHI) ? K.spec_hi : K.spec_pore);
                wall = (M::uniform(r.y) < p) ? (int)LE_MC_WALL_SPECULAR : (int)LE_MC_WALL_DIFFUSE;
            }
        }
        // a film whose walls are all diffuse: every hit is a diffuse wall
        constexpr bool FILM_DIFF = DIFF && GEOM == LE_MC_GEOM_PLANES;
        const bool on_wall = FILM_DIFF ? hit : wall >= 0;
        const bool absorbed = FILM_DIFF ? false : wall == LE_MC_WALL_BLACK;
        const bool diffuse = FILM_DIFF ? hit : wall == LE_MC_WALL_DIFFUSE;
        const bool periodic = FILM_DIFF ? false : hit && !on_wall;
        // Eq. 2 redraw (kept only on a relaxation event)
        if constexpr (FUSED) {
            const unsigned long long mm = (unsigned long long)r.y * (uint32_t)n_modes;
            const uint4 e = s_fused[(uint32_t)(mm >> 32)];
            const R lam_new = __uint_as_float(((uint32_t)mm < e.x) ? e.z : e.w);
            lam = scat ? lam_new : lam;
        } else {
            uint32_t m_new = alias_draw(s_scat, (uint32_t)n_modes, r.y);
            LEMC_GUARD_INDEX(m_new, n_modes);
            const R lam_new = s_props[2 * m_new], vg_new = s_props[2 * m_new + 1];
            lam = scat ? lam_new : lam;
            vg = scat ? vg_new : vg;
        }
        // fresh direction: isotropic (relaxation) or Lambertian (diffuse wall)
        const R u2 = M::uniform(r.z);
        R sn, cs;
        M::sincos_2pi(M::uniform(r.w), &sn, &cs);
        const R mu = scat ? (R(2) * u2 - R(1)) : M::sqrt_(u2);
        const R st = M::sqrt_(fmax(R(0), R(1) - mu * mu));
        const R a = st * cs, b = st * sn;
        // direction after a relaxation: isotropic (a, b, mu) about z, or the
        // Henyey-Greenstein law of mean cosine g about the incoming direction,
        // its cosine from the inverted CDF and its azimuth in the
        // orthonormal frame of Duff et al. (JCGT 2017) built on (ox, oy, oz)
        R sx = a, sy = b, sz = mu;
        if (aniso && scat) {
            const R q = M::div(R(1) - hg * hg, R(1) - hg + R(2) * hg * u2);
            R mh = M::div(R(1) + hg * hg - q * q, R(2) * hg);
            mh = fmin(fmax(mh, R(-1)), R(1));
            const R sh = M::sqrt_(fmax(R(0), R(1) - mh * mh));
            const R sg = oz >= R(0) ? R(1) : R(-1);
            const R fa = M::div(R(-1), sg + oz);
            const R fb = ox * oy * fa;
            sx = mh * ox + sh * (cs * (R(1) + sg * ox * ox * fa) + sn * fb);
            sy = mh * oy + sh * (cs * (sg * fb) + sn * (sg + oy * oy * fa));
            sz = mh * oz + sh * (cs * (-sg * ox) + sn * (-oy));
        }
        R nox = sx, noy = sy, noz = sz;
        if constexpr (GEOM != LE_MC_GEOM_BULK) {
            // x walls: Lambertian about +-x, or mirror
            const R wox = diffuse ? ((kind == HIT_XLO) ? mu : -mu) : -ox;
            const R woy = diffuse ? a : oy;
            const R woz = diffuse ? b : oz;
            if constexpr (POROUS) {
                // pore wall: normal from the axis to the hit point
                const R ny = (y - half) / rad, nz = (z - half) / rad;
                const R dn = oy * ny + oz * nz;
                const R cox = diffuse ? a : ox;
                const R coy = diffuse ? (mu * ny - b * nz) : (oy - R(2) * dn * ny);
                const R coz = diffuse ? (mu * nz + b * ny) : (oz - R(2) * dn * nz);
                const bool cyl = kind == HIT_CYL;
                nox = scat ? sx : (periodic ? ox : (cyl ? cox : wox));
                noy = scat ? sy : (periodic ? oy : (cyl ? coy : woy));
                noz = scat ? sz : (periodic ? oz : (cyl ? coz : woz));
                // periodic unit-cell face: re-insert on the opposite face
                const bool yhi = periodic && kind == HIT_YHI, ylo = periodic && kind == HIT_YLO;
                const bool zhi = periodic && kind == HIT_ZHI, zlo = periodic && kind == HIT_ZLO;
                y = yhi ? R(0) : (ylo ? pitch : y);
                z = zhi ? R(0) : (zlo ? pitch : z);
                // unit-cell indices wrapped into the periodic domain (only the
                // transient grid needs them)
                if constexpr (TRANSIENT) {
                    cy = yhi ? (cy + 1 == P.cells_y ? 0 : cy + 1) : (ylo ? (cy == 0 ? P.cells_y - 1 : cy - 1) : cy);
                    cz = zhi ? (cz + 1 == P.cells_z ? 0 : cz + 1) : (zlo ? (cz == 0 ? P.cells_z - 1 : cz - 1) : cz);
                }
            } else {
                nox = scat ? sx : wox;
                noy = scat ? sy : woy;
                noz = scat ? sz : woz;
            }
        }
        ox = nox;
        oy = noy;
        oz = noz;
        // (every segment ends in exactly one of a relaxation event, a wall
        // and a periodic face, so the wall count is n_seg - n_scat - n_per,
        // formed when the particle ends)
        n_scat += scat ? 1u : 0u;
        n_per += periodic ? 1u : 0u;
        if constexpr (HJ) {  // flux split by scattering index
            if (P.n_hj > 0 && scat) {
                if (n_scat - 1u < (uint32_t)P.n_hj) {
                    red64(&P.hj[n_scat - 1u], (R)sign * hrun);
                    red64(&P.hj[P.n_hj + n_scat - 1u], hrun * hrun);
                }
                hrun = R(0);
            }
        }
        // step VI and truncation: one combined test per segment; the fate
        // (first reason in the order absorption, t_final, scattering cap,
        // collision cap, segment cap) is only worked out when the particle ends
        const bool t_out = TRANSIENT && t > K.t_final;
        const bool s_cap = n_scat >= P.scat_cap;  // scat_cap = max_scatter, or 2^32 - 1 for none
        const bool c_cap = col_cap && n_seg - n_per >= P.max_collisions;  // relaxation events + wall hits
        if (absorbed || t_out || s_cap || c_cap || n_seg >= P.max_events) {
            fate = absorbed ? FATE_ABSORBED
                 : t_out    ? FATE_T_FINAL
                 : s_cap    ? FATE_MAX_SCATTER
                 : c_cap    ? FATE_MAX_COLLISIONS
                            : FATE_MAX_EVENTS;
            alive = false;
            pending = true;
        }
    };

    // totals of a finished particle (step V, Eq. 4) into the lane accumulators
    auto finish = [&]() {
        n_wall = n_seg - n_scat - n_per;
        if constexpr (BATCH) {
            if (bidx != cur_b) {
                flush_lane(cur_b);
                cur_b = bidx;
            }
        }
        const R sL = (R)sign * Lacc;
        const uint32_t trunc =
            (fate == FATE_MAX_SCATTER || fate == FATE_MAX_EVENTS || fate == FATE_MAX_COLLISIONS) ? 1u : 0u;
        const uint32_t absd = (fate == FATE_ABSORBED) ? 1u : 0u;
        if constexpr (LANE_SMEM) {
            Acc<R> a0, a1;
            a0.s = __uint_as_float(lt[0]);
            a0.c = __uint_as_float(lt[lts]);
            a1.s = __uint_as_float(lt[2 * lts]);
            a1.c = __uint_as_float(lt[3 * lts]);
            a0.add(sL);
            a1.add(sL * sL);
            lt[0] = __float_as_uint(a0.s);
            lt[lts] = __float_as_uint(a0.c);
            lt[2 * lts] = __float_as_uint(a1.s);
            lt[3 * lts] = __float_as_uint(a1.c);
            lt[4 * lts] += 1u;
            lt[5 * lts] += n_seg;
            lt[6 * lts] += n_scat;
            lt[7 * lts] += n_wall;
            lt[8 * lts] += n_per;
            lt[9 * lts] += trunc;
            lt[10 * lts] += absd;
        } else {
            acc_sL.add(sL);
            acc_sL2.add(sL * sL);
            c_part += 1;
            c_seg += n_seg;
            c_scat += n_scat;
            c_wall += n_wall;
            c_per += n_per;
            c_trunc += trunc;
            c_abs += absd;
        }
        if (HJ && P.n_hj > 0 && n_scat < (uint32_t)P.n_hj && hrun != R(0)) {
            red64(&P.hj[n_scat], (R)sign * hrun);
            red64(&P.hj[P.n_hj + n_scat], hrun * hrun);
        }
        if (P.records) {
            le_mc_particle rec;
            rec.sign = (int8_t)sign;
            rec.fate = (int8_t)(fate == FATE_MAX_EVENTS ? P.events_fate : fate);  // a folded collision cap
            rec.pad = 0;
            rec.n_seg = n_seg;
            rec.n_scat = n_scat;
            rec.n_wall = n_wall;
            rec.n_periodic = n_per;
            rec.mode0 = mode0;
            rec.L_axis = (double)Lacc;
            rec.x0 = (double)x0;
            rec.t0 = (double)t0;
            uint32_t ri = pid - P.first;
            LEMC_GUARD_INDEX(ri, P.n_particles);
            P.records[ri] = rec;
        }
        pending = false;
    };

    // Rounds of precomputed random words, for a warp tracing one extreme
    // particle (phase A): such a warp runs at the latency of one lane, so its
    // idle lanes compute the particle's next random words (the counters are
    // known in advance) into the emission buffer's storage, and the particle
    // traces a round of segments without Philox on its critical path.  Each
    // segment uses the same words as otherwise.
    //
    // Reproducibility: the rounds inline a second copy of the segment code,
    // whose FP32 operations the compiler may contract differently from the
    // main loop's copy, so a particle must always be traced by the same copy.
    // The set of extreme particles is fixed by their emission modes (and is
    // used all or nothing, see n_ext), so which copy traces a particle never
    // depends on timing, and results are bit-identical across runs and
    // launch shapes.  (Assisting whichever lanes happen to be last at the end
    // of the queue broke that and is not done.)
    auto assisted = [&]() {
        uint4* const words = reinterpret_cast<uint4*>(&buf);
        for (;;) {
            const unsigned m = __ballot_sync(FULL, alive);
            if (m == 0) break;
            const int n_a = __popc(m);
            const int steps = 32 / n_a;
            const int a = lane % n_a, s = lane / n_a;
            unsigned mm = m;
            for (int i = 0; i < a; ++i) mm &= mm - 1u;
            const int src = __ffs((int)mm) - 1;
            const uint32_t seg_a = __shfl_sync(FULL, n_seg, src);
            const uint32_t pid_a = __shfl_sync(FULL, pid, src);
            const uint32_t inst_a = __shfl_sync(FULL, instw, src);
            if (s < steps) words[s * n_a + a] = philox4x32_10(make_uint4(seg_a + 1u + (uint32_t)s, 0u, pid_a, inst_a), rk);
            __syncwarp();
            if (alive) {
                const int my = __popc(m & lanemask_lt);
                for (int k = 0; k < steps && alive; ++k) segment(words[k * n_a + my], false);
            }
            __syncwarp();
            if (pending) finish();
        }
    };

    // step I for queue position `pos` (a particle id of the run, or a position
    // in the concatenated instances of a batch) into emission-buffer slot
    // base + popc(before): the slot is formed after the emission, which keeps
    // it out of the registers live across emit_particle
    auto emit_to = [&](uint32_t pos, int base, unsigned before) {
        uint32_t id = pos, eb = 0;
        EmitCtx<R> ctx;
        if constexpr (BATCH) {
            eb = batch_find(P.offsets, (uint32_t)P.n_instances, pos);
            LEMC_GUARD_INDEX(eb, P.n_instances);
            id = (uint32_t)(pos - P.offsets[eb]);
            ctx = batch_ctx<R>(P.instances[eb]);
        } else {
            id = P.first + pos;
            ctx = run_ctx<R>(P);
        }
        R ex, ey, ez, eox, eoy, eoz, et;
        uint32_t em, ecy, ecz;
        int es;
        if (!emit_particle<R, GEOM, SRC>(P, ctx, rk, SRC == LE_MC_SRC_INITIAL ? P.alias_init : P.alias_emit, id, ex, ey,
                                         ez, eox, eoy, eoz, et, em, es, ecy, ecz))
            flags |= FLAG_REJECTION_EXHAUSTED;
        int slot = base + __popc(before);
        LEMC_GUARD_INDEX(slot, kBufSlots);
        buf.x[slot] = ex;
        buf.ox[slot] = eox;
        buf.oy[slot] = eoy;
        buf.oz[slot] = eoz;
        buf.pid[slot] = id;
        buf.mode_sign[slot] = em | (es < 0 ? 0x80000000u : 0u);
        if constexpr (POROUS) {
            buf.y.v[slot] = ey;
            buf.z.v[slot] = ez;
            buf.cell.v[slot] = ecy | (ecz << 16);
        }
        if constexpr (SRC == LE_MC_SRC_PULSE) buf.t.v[slot] = et;
        if constexpr (BATCH) buf.inst.v[slot] = eb;
    };

    // start this lane's next particle from emission-buffer slot `slot`
    auto take = [&](int slot) {
        LEMC_GUARD_INDEX(slot, kBufSlots);
        x = buf.x[slot];
        ox = buf.ox[slot];
        oy = buf.oy[slot];
        oz = buf.oz[slot];
        pid = buf.pid[slot];
        const uint32_t ms = buf.mode_sign[slot];
        if constexpr (POROUS) {
            y = buf.y.v[slot];
            z = buf.z.v[slot];
            const uint32_t cell = buf.cell.v[slot];
            cy = (int)(cell & 0xFFFFu);
            cz = (int)(cell >> 16);
        }
        if constexpr (SRC == LE_MC_SRC_PULSE) t = buf.t.v[slot];
        if constexpr (SRC == LE_MC_SRC_INITIAL) t = R(0);
        if constexpr (BATCH) {
            bidx = buf.inst.v[slot];
            const BatchInstance& bi = P.instances[bidx];
            if constexpr (sizeof(R) == 4) Lp = bi.L32;
            else Lp = bi.L;
            instw = bi.inst_id;
        }
        mode0 = ms & 0x7FFFFFFFu;
        LEMC_GUARD_INDEX(mode0, n_modes);
        if constexpr (PROFILE) {
            // batch group of the error bars: particle ids mod n_batch, or
            // particle pairs (2i, 2i + 1) for the gradient source, whose even
            // and odd ids carry opposite signs (every group holds both signs)
            pgroup = AXIS_X ? (int)((pid - P.first) % (uint32_t)P.n_batch)
                            : (int)(((pid - P.first) >> 1) % (uint32_t)P.n_batch);
        }
        sign = (ms >> 31) ? -1 : 1;
        if constexpr (FUSED) {
            lam = __uint_as_float(s_fused[mode0].z);
        } else {
            lam = s_props[2 * mode0];
            vg = s_props[2 * mode0 + 1];
        }
        plane = philox_lane(pid, instw, rk);
        x0 = x;
        t0 = t;
        Lacc = 0;
        hrun = 0;
        n_seg = n_scat = n_per = 0;
        alive = true;
    };

    // Phase A: extreme particles, one per otherwise empty warp, claimed first.
    if (n_ext > 0) {
        for (;;) {
            unsigned int e = 0;
            if (lane == 0) e = atomicAdd(P.long_count + 2, 1u);
            e = __shfl_sync(FULL, e, 0);
            if (e >= n_ext) break;
            if (lane == 0) {  // lane 0 starts it from the buffer, as a refill would
                emit_to(P.long_list[e], 0, 0u);
                take(0);
            }
            __syncwarp();
            assisted();
        }
    }

    // Phase B: the queue (long-first list, then the natural order).
    for (;;) {
        if constexpr (TRANSIENT) flush_jobs();
        if constexpr (PROFILE && POROUS) flush_map_jobs();
        if (PROF32 && prof32_len > 0 && ++drain_it == kProfDrainEvery) {
            drain_it = 0;
            const int per = (prof32_len + n_warps - 1) / n_warps;
            const int w = (int)(threadIdx.x >> 5);
            drain_prof(w * per, min((w + 1) * per, prof32_len));
        }
        const unsigned dead = __ballot_sync(FULL, !alive);
        // refill once refill_min lanes are idle (or at once near the end)
        if (dead && (dead == FULL || qdone || __popc(dead) >= refill_min)) {
            if (pending) finish();
            const int need = __popc(dead);
            while (cnt < need && !qdone) {
                uint32_t pos = 0;
                bool valid = false;
                // step I for the next 32 claimed queue positions, whole warp
                if (w_next >= w_end) {
                    unsigned long long base = 0;
                    const unsigned long long claim = (w_end < n_long) ? long_claim : chunk;
                    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(P.queue), claim);
                    base = __shfl_sync(FULL, base, 0);
                    w_next = base;
                    w_end = min(base + claim, q_total);
                    if (base >= q_total) {
                        qdone = true;
                        break;
                    }
                }
                const unsigned long long q = w_next + (unsigned long long)lane;
                const unsigned long long q_end = w_end;
                w_next = min(w_next + 32ull, w_end);
                if (w_next >= w_end && w_end >= q_total) qdone = true;
                if (q >= q_end) {
                    valid = false;
                } else if (q < n_long) {
                    pos = long_region[q];
                    LEMC_GUARD_INDEX(pos, n_pos);
                    valid = true;
                } else {
                    pos = (uint32_t)(q - n_long);
                    valid = !(P.long_list && ((P.long_bits[pos >> 5] >> (pos & 31u)) & 1u));
                }
                const unsigned vmask = __ballot_sync(FULL, valid);
                if (valid) emit_to(pos, cnt, vmask & lanemask_lt);
                cnt += __popc(vmask);
                __syncwarp();
            }
            if (!alive) {
                const int rank = __popc(dead & lanemask_lt);
                if (rank < cnt) take(cnt - 1 - rank);
            }
            cnt -= min(cnt, need);
            __syncwarp();
            if (!__any_sync(FULL, alive)) break;  // queue exhausted and buffer empty
        }
        if (!alive) continue;
        if constexpr (SRC == LE_MC_SRC_GRADIENT && !(PROFILE && POROUS)) {
            // Kernels of the gradient source (long histories) without deferred
            // per-warp jobs trace up to 2 x kFlightPairs segments per
            // iteration: the loop's refill test runs that much less often, and
            // the random words of each pair of flights are formed together
            // ahead of them (the counters are known in advance), two
            // independent Philox chains whose latencies overlap.  The words of
            // a flight the particle does not live to take are discarded.
            // (1e7-particle film, trace kernel: 1, 2, 3, 4, 6, 8, 10, 12
            // flights per iteration 2.84, 2.56, 2.40, 2.32, 2.25, 2.21, 2.20,
            // 2.23 ms; the 2e7-particle pored film 13.0 ms at 4 and 8, 12.9
            // at 6.  For the short histories of the walls source a second
            // flight measured slower.)  The pairs are unrolled, and
            // every particle starts at the top of the loop, so its segment k
            // always runs in copy k mod (2 kFlightPairs) of the segment code:
            // which copy traces a segment never depends on timing.
            constexpr int kFlightPairs = POROUS ? 3 : 4;
#pragma unroll
            for (int pr = 0; pr < kFlightPairs; ++pr) {
                if (pr > 0 && !alive) break;
                const uint4 ra = philox_flight(n_seg + 1u, plane, rk);
                const uint4 rb = philox_flight(n_seg + 2u, plane, rk);
                segment(ra, true);
                if (alive) segment(rb, true);
            }
        } else {
            segment(philox_flight(n_seg + 1u, plane, rk), true);
        }
    }
    if constexpr (TRANSIENT) flush_jobs();
    if constexpr (PROFILE && POROUS) flush_map_jobs();

    // ---- flush: warp shuffles, then one FP64 / u64 atomic per quantity ----
    if constexpr (BATCH) {
        flush_lane(cur_b);
        const uint32_t fl = __reduce_or_sync(FULL, flags);
        if (lane == 0 && fl) atomicOr(P.flags, fl);
        if (inst_len > 0) {
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * inst_len; i += blockDim.x)
                if (s_isum[i] != 0.0) atomicAdd(&P.inst_sums[i], s_isum[i]);
            for (int i = threadIdx.x; i < CNT_N * inst_len; i += blockDim.x)
                if (s_icnt[i]) atomicAdd(&P.inst_counters[i], s_icnt[i]);
        }
        return;
    }
    if (PROF32 && prof32_len > 0) {  // what the warps have not drained yet
        __syncthreads();
        for (int i = threadIdx.x; i < prof32_len; i += blockDim.x)
            if (s_prof32[i] != 0.0f) red64(P.prof + i, (R)s_prof32[i]);
    }
    if constexpr (LANE_SMEM) {
        acc_sL.s = __uint_as_float(lt[0]);
        acc_sL.c = __uint_as_float(lt[lts]);
        acc_sL2.s = __uint_as_float(lt[2 * lts]);
        acc_sL2.c = __uint_as_float(lt[3 * lts]);
        c_part = lt[4 * lts];
        c_seg = lt[5 * lts];
        c_scat = lt[6 * lts];
        c_wall = lt[7 * lts];
        c_per = lt[8 * lts];
        c_trunc = lt[9 * lts];
        c_abs = lt[10 * lts];
    }
    double v0 = acc_sL.value(), v1 = acc_sL2.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(FULL, v0, o);
        v1 += __shfl_xor_sync(FULL, v1, o);
    }
    unsigned long long red[CNT_N] = {c_part, c_seg, c_scat, c_wall, c_per, c_trunc, c_abs};
#pragma unroll
    for (int i = 0; i < CNT_N; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) red[i] += __shfl_xor_sync(FULL, red[i], o);
    const uint32_t fl = __reduce_or_sync(FULL, flags);
    if (lane == 0) {
        atomicAdd(&P.sums[0], v0);
        atomicAdd(&P.sums[1], v1);
#pragma unroll
        for (int i = 0; i < CNT_N; ++i)
            if (red[i]) atomicAdd(&P.counters[i], red[i]);
        if (fl) atomicOr(P.flags, fl);
    }
}

// Kernel entry points.  Some FP32 kernels are held to 64 registers (two
// 512-thread blocks per SM) although that spills: measured on GB300, the
// doubled occupancy outweighs the spills for the pored-film kernels (steady
// pored film +7 %, surface pulse +17 %; ~250 bytes of spills per thread) and
// for the kernels whose tallies go through memory (slab profiles, steady
// maps), whose registers would otherwise allow one block per SM.  The others
// keep the compiler's own register choice (naming a minimum of one block
// changes it for the worse).
template <typename R, int GEOM, int SRC, bool PROFILE, bool BATCH = false, bool DIFF = false>
__global__ void __launch_bounds__(512) trace_kernel(const __grid_constant__ KernelArgs args)
{
    trace_body<R, GEOM, SRC, PROFILE, BATCH, DIFF>(args);
}

template <typename R, int GEOM, int SRC, bool PROFILE, bool DIFF = false>
__global__ void __launch_bounds__(512, 2) trace_kernel_2b(const __grid_constant__ KernelArgs args)
{
    trace_body<R, GEOM, SRC, PROFILE, false, DIFF>(args);
}

// FP32 kernels of the gradient source that trace two flights per loop
// iteration (films, plain and batched, and the steady pored film), which want
// ~90 registers, and the pored film's steady maps: held to 80, which keeps
// three 256-thread blocks per SM instead of two (film: no spills, 2 % faster
// than the compiler's choice and 4 % faster than 64 registers with spills;
// pored film: 60 bytes of spills instead of 270 at 64 registers, 3.6 %
// faster; maps: 4.5 % faster).
template <typename R, int GEOM, int SRC, bool PROFILE, bool BATCH = false, bool DIFF = false>
__global__ void __maxnreg__(80) trace_kernel_r80(const __grid_constant__ KernelArgs args)
{
    trace_body<R, GEOM, SRC, PROFILE, BATCH, DIFF>(args);
}

// The entry point of a configuration.
template <typename R, int GEOM, int SRC, bool PROFILE, bool BATCH = false, bool DIFF = false>
constexpr auto trace_entry()
{
    if constexpr (sizeof(R) == 4 && SRC == LE_MC_SRC_GRADIENT && (!PROFILE || GEOM == LE_MC_GEOM_POROUS) &&
                  (GEOM == LE_MC_GEOM_PLANES || (GEOM == LE_MC_GEOM_POROUS && !BATCH)))
        return trace_kernel_r80<R, GEOM, SRC, PROFILE, BATCH, DIFF>;
    else if constexpr (sizeof(R) == 4 && !BATCH && (GEOM == LE_MC_GEOM_POROUS || PROFILE))
        return trace_kernel_2b<R, GEOM, SRC, PROFILE, DIFF>;
    else
        return trace_kernel<R, GEOM, SRC, PROFILE, BATCH, DIFF>;
}

// Long-first schedule, pass 1: flag the particles whose emission mode has a
// mean free path above lam_cut (they make the longest trajectories: many
// wall segments before their first relaxation event) and list them so the
// trace kernel can serve them first; those above kExtremeFactor x lam_cut go
// to the extreme list (traced one per warp in phase A) while it has room.
// Same random words as step I.
template <typename R>
__global__ void __launch_bounds__(256) classify_kernel(const __grid_constant__ KernelArgs args)
{
    const TraceParams& P = args.p;
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const bool batch = P.instances != nullptr;
    // N may reach 2^32 - 1: the loop index and the bound test are 64-bit, so
    // neither w0 + stride nor w0 + lane can wrap around below N
    const unsigned long long N = batch ? P.offsets[P.n_instances] : (unsigned long long)P.n_particles;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // whole warps iterate together so the ballots below see full masks
    const unsigned long long first = (unsigned long long)((blockIdx.x * blockDim.x + threadIdx.x) & ~31u);
    for (unsigned long long w0 = first; w0 < N; w0 += stride) {
        const unsigned long long pid64 = w0 + (unsigned long long)lane;
        const uint32_t pid = (uint32_t)pid64;
        bool is_long = false, is_ext = false;
        if (pid64 < N) {
            uint32_t id = batch ? pid : P.first + pid, inst = P.inst;
            R cut = consts_of<R>(P).lam_cut;
            if (batch) {
                const uint32_t b = batch_find(P.offsets, (uint32_t)P.n_instances, pid);
                id = (uint32_t)(pid - P.offsets[b]);
                inst = P.instances[b].inst_id;
                if constexpr (sizeof(R) == 4) cut = P.instances[b].lam_cut32;
                else cut = P.instances[b].lam_cut;
            }
            const uint4 r = philox4x32_10(make_uint4(0u, 0u, id, inst), args.rk);
            const uint2* table = P.src == LE_MC_SRC_INITIAL ? P.alias_init : P.alias_emit;
            const uint32_t mode = alias_draw(table, (uint32_t)P.n_modes, r.y);
            R lam, vg;
            load_props<R>(P.props, mode, lam, vg);
            is_long = lam > cut;
            is_ext = lam > cut * R(kExtremeFactor);
        }
        // extreme particles first (while the extreme list has room)
        bool listed = false;
        const unsigned mx = __ballot_sync(FULL, is_ext);
        if (mx && P.ext_cap > 0) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(P.long_count + 1, (unsigned)__popc(mx));
            base = __shfl_sync(FULL, base, 0);
            if (is_ext) {
                const unsigned slot = base + (unsigned)__popc(mx & lanemask_lt);
                if (slot < P.ext_cap) {
                    P.long_list[slot] = pid;
                    atomicOr(&P.long_bits[pid >> 5], 1u << (pid & 31u));
                    listed = true;
                }
            }
        }
        const bool to_long = is_long && !listed;
        const unsigned m = __ballot_sync(FULL, to_long);
        if (m) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(P.long_count, (unsigned)__popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (to_long) {
                const unsigned slot = base + (unsigned)__popc(m & lanemask_lt);
                if (slot < P.long_cap) {
                    P.long_list[P.ext_cap + slot] = pid;
                    atomicOr(&P.long_bits[pid >> 5], 1u << (pid & 31u));
                }
            }
        }
    }
}

// Dynamic shared memory of one block.
template <typename R, int GEOM, int SRC, bool PROFILE, bool BATCH = false>
inline size_t trace_smem_bytes(int n_modes, int threads, int prof_len, int hj_len, int n_instances = 0)
{
    size_t off = table_bytes<R, SRC, PROFILE>(n_modes);
    off += (size_t)(threads / 32) * sizeof(BufferOf<R, GEOM, SRC, BATCH>);
    if (SRC == LE_MC_SRC_PULSE || SRC == LE_MC_SRC_INITIAL) off += (size_t)(threads / 32) * sizeof(SampleJobs<R>);
    if (PROFILE && GEOM == LE_MC_GEOM_POROUS) off += (size_t)(threads / 32) * sizeof(MapJobs<R>);
    // prof_len: entries of the FP32 shared-memory copy of the slab profile or
    // steady maps (0 = none); the H_j split is reduced in global memory
    if (PROFILE && sizeof(R) == 4) off += (size_t)prof_len * sizeof(float);
    off = (off + 7) & ~(size_t)7;
    (void)hj_len;
    if (BATCH && n_instances <= kBatchSmemMax)
        off += (size_t)n_instances * (2 * sizeof(double) + CNT_N * sizeof(unsigned long long));
    if (LaneTallyInSmem<R, GEOM, SRC, PROFILE, BATCH>::value) off += (size_t)threads * kLaneWords * sizeof(uint32_t);
    return off;
}

}  // namespace lemc
