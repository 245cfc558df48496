// Resident trace kernel of the request server (le_mc_server_*).
//
// Not in the paper: the method's steps I-VI for many independent simulation
// requests, interleaved inside one long-running persistent kernel.  The host
// keeps each admitted request in a slot whose parameters (ServeSlot: the run's
// TraceParams, its Philox round keys and its Eq. 2 table) and tallies
// (ServeTally) stay in device memory from admission to retirement, and appends
// work items (slot, first particle id, count) to a ring in mapped host memory.
// Every warp of the kernel claims one item at a time (compare-and-swap on a
// device head counter, after reading the published tail with acquire
// semantics) and traces that item's particles of that request: emission by the
// library's step I (emit_particle), then flights, boundary search, wall or
// relaxation handling and the Eq. 4 path sum, all with the request's own
// geometry and material.  Items of different requests, geometries and
// materials therefore run side by side on the GPU.  At the end of an item the
// warp adds its sums and counters to the slot's tallies and then, after a
// fence, the item's particle count to the slot's `done` counter, which is what
// the host polls.
//
// Waits are bounded: a warp that finds no published item sleeps in steps of
// a few microseconds and leaves the kernel when the ring's stop word is set,
// when it has found no work for `idle_ns` nanoseconds (%globaltimer), or after
// kMaxPolls polls; the host relaunches the kernel when work arrives after it
// has left.  Nothing waits on another warp or another kernel.
#include <cuda_runtime.h>

#include "le_mc_internal.h"
#include "trace_kernel.cuh"
#include "serve_kernel.h"

namespace lemc {

namespace {

constexpr unsigned kMaxPolls = 1u << 22;  // hard limit of one warp's wait for work
constexpr unsigned kSleepNs = 2000;       // one sleep between polls

__device__ __forceinline__ unsigned long long load_acquire_sys(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned load_acquire_sys(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Emission buffer of one warp: step I for 32 particles at a time, run by the
// whole warp (converged), and popped by the lanes whose particle has ended.
struct ServeBuf {
    float x[64], y[64], z[64], ox[64], oy[64], oz[64], lam[64];
    uint32_t pid[64];
    int32_t sign[64];
};

// One work item of family (GEOM, SRC) traced by the whole warp: particle ids
// first .. first + count - 1 of the request in slot S.  Lanes trace one
// particle each; once at least kRefill lanes are idle (or the item is running
// out) the warp emits the next 32 ids together into its buffer and the idle
// lanes take particles from it, as in the run kernels.  FP32
// trajectories as in the run kernels (same random-word layout, frames and
// rules, so a particle follows the same kind of history it has in le_mc_run),
// compensated FP32 per-lane sums, FP64 accumulation across lanes.
template <int GEOM, int SRC>
__device__ void serve_item(const ServeSlot& S, ServeTally& T, ServeBuf& buf, uint32_t first, uint32_t count)
{
    using R = float;
    using M = DMath<R>;
    constexpr bool POROUS = GEOM == LE_MC_GEOM_POROUS;
    constexpr bool AXIS_X = SRC == LE_MC_SRC_WALLS;
    constexpr int kRefill = 4;
    // the request's round keys in registers (read by every flight)
    const RoundKeys rk = S.rk;
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const TraceParams& P = S.p;
    const Consts<R>& K = P.c32;
    const EmitCtx<R> ctx = run_ctx<R>(P);
    // warp-uniform problem constants, in registers for the item
    const R Lp = K.L, pitch = K.pitch, half = K.half, rad = K.rad, rad2 = K.rad2;
    const int wall_lo = P.wall_lo, wall_hi = P.wall_hi, pore_wall = P.pore_wall;
    const uint32_t scat_cap = P.scat_cap, max_events = P.max_events, max_col = P.max_collisions;
    const bool col_cap = POROUS && max_col > 0u;
    const uint32_t n_modes = (uint32_t)P.n_modes;
    const uint4* fused = S.fused;
    const uint2* alias_emit = P.alias_emit;
    const uint32_t inst = P.inst;
    const R big = M::big();

    R x = 0, y = 0, z = 0, ox = 0, oy = 0, oz = 1, lam = 1, Lacc = 0;
    uint32_t n_seg = 0, n_scat = 0, n_wall = 0, n_per = 0;
    int sign = 1, fate = FATE_MAX_EVENTS;
    bool alive = false, pending = false;
    PhiloxLane pl = {0u, 0u, 0u};
    Acc<R> acc_sL, acc_sL2;
    uint32_t c_part = 0, c_seg = 0, c_scat = 0, c_wall = 0, c_per = 0, c_trunc = 0, c_abs = 0, flags = 0;

    auto finish = [&]() {
        const R sL = (R)sign * Lacc;
        acc_sL.add(sL);
        acc_sL2.add(sL * sL);
        c_part += 1;
        c_seg += n_seg;
        c_scat += n_scat;
        c_wall += n_wall;
        c_per += n_per;
        c_trunc += (fate == FATE_MAX_SCATTER || fate == FATE_MAX_EVENTS || fate == FATE_MAX_COLLISIONS) ? 1u : 0u;
        c_abs += (fate == FATE_ABSORBED) ? 1u : 0u;
        pending = false;
    };

    // steps II-VI for one flight, from its four random words
    auto step = [&](const uint4 r) {
        // step II: -Lambda ln u with the table's Lambda ln 2 and log2
        const R ell = -(lam * __log2f(M::uniform(r.x)));
        // step III: first boundary along the ray
        R d_b = big;
        int kind = HIT_NONE;
        if constexpr (GEOM != LE_MC_GEOM_BULK) {
            const bool up = ox > R(0);
            d_b = M::div(up ? (Lp - x) : x, fabs(ox));
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
            const R tfy = M::div(oy > R(0) ? pitch - y : y, fabs(oy));
            if (tfy < d_b) { d_b = tfy; kind = oy > R(0) ? HIT_YHI : HIT_YLO; }
            const R tfz = M::div(oz > R(0) ? pitch - z : z, fabs(oz));
            if (tfz < d_b) { d_b = tfz; kind = oz > R(0) ? HIT_ZHI : HIT_ZLO; }
        }
        bool hit = (kind != HIT_NONE) && (d_b <= ell);
        if constexpr (SRC == LE_MC_SRC_WALLS && GEOM == LE_MC_GEOM_PLANES) {
            // absorbing walls decide a fate: near ties are redone in FP64
            const int wt = (kind == HIT_XLO) ? wall_lo : wall_hi;
            if (wt == LE_MC_WALL_BLACK && fabsf(d_b - ell) <= 8.0f * 1.1920929e-7f * fmaxf(d_b, ell)) {
                const double u = (double)M::uniform(r.x);
                const double ell64 = (double)lam * (-log2(u));
                const double d64 = ((ox > 0.0f) ? ((double)Lp - (double)x) : (double)x) / fabs((double)ox);
                hit = d64 <= ell64;
            }
        }
        R seg = hit ? d_b : ell;
        if constexpr (SRC == LE_MC_SRC_WALLS && GEOM == LE_MC_GEOM_PLANES) seg = hit ? d_b : fminf(ell, d_b);
        R x_new = x + ox * seg;
        if (hit && kind == HIT_XLO) x_new = R(0);
        if (hit && kind == HIT_XHI) x_new = Lp;
        // step V: the Eq. 4 path sum along the flux axis
        Lacc += AXIS_X ? (x_new - x) : oz * seg;
        x = x_new;
        if constexpr (POROUS) {
            y += oy * seg;
            z += oz * seg;
        }
        ++n_seg;
        // steps IVa / IVb
        const bool scat = !hit;
        int wall = (kind == HIT_XLO) ? wall_lo : ((kind == HIT_XHI) ? wall_hi : -1);
        if constexpr (POROUS) wall = (kind == HIT_CYL) ? pore_wall : wall;
        wall = hit ? wall : -1;
        const bool on_wall = wall >= 0;
        const bool absorbed = wall == LE_MC_WALL_BLACK;
        const bool diffuse = wall == LE_MC_WALL_DIFFUSE;
        const bool periodic = hit && !on_wall;
        // Eq. 2 redraw of the mode (kept only on a relaxation event)
        {
            const unsigned long long mm = (unsigned long long)r.y * n_modes;
            const uint4 e = fused[(uint32_t)(mm >> 32)];
            const R lam_new = __uint_as_float(((uint32_t)mm < e.x) ? e.z : e.w);
            lam = scat ? lam_new : lam;
        }
        const R u2 = M::uniform(r.z);
        R sn, cs;
        M::sincos_2pi(M::uniform(r.w), &sn, &cs);
        const R mu = scat ? (R(2) * u2 - R(1)) : M::sqrt_(u2);
        const R st = M::sqrt_(fmax(R(0), R(1) - mu * mu));
        const R a = st * cs, b = st * sn;
        R nox = a, noy = b, noz = mu;  // relaxation: isotropic about z
        if constexpr (GEOM != LE_MC_GEOM_BULK) {
            const R wox = diffuse ? ((kind == HIT_XLO) ? mu : -mu) : -ox;
            const R woy = diffuse ? a : oy;
            const R woz = diffuse ? b : oz;
            if constexpr (POROUS) {
                const R ny = (y - half) / rad, nz = (z - half) / rad;
                const R dn = oy * ny + oz * nz;
                const R cox = diffuse ? a : ox;
                const R coy = diffuse ? (mu * ny - b * nz) : (oy - R(2) * dn * ny);
                const R coz = diffuse ? (mu * nz + b * ny) : (oz - R(2) * dn * nz);
                const bool cyl = kind == HIT_CYL;
                nox = scat ? a : (periodic ? ox : (cyl ? cox : wox));
                noy = scat ? b : (periodic ? oy : (cyl ? coy : woy));
                noz = scat ? mu : (periodic ? oz : (cyl ? coz : woz));
                // periodic unit-cell face: re-insert on the opposite face
                y = (periodic && kind == HIT_YHI) ? R(0) : ((periodic && kind == HIT_YLO) ? pitch : y);
                z = (periodic && kind == HIT_ZHI) ? R(0) : ((periodic && kind == HIT_ZLO) ? pitch : z);
            } else {
                nox = scat ? a : wox;
                noy = scat ? b : woy;
                noz = scat ? mu : woz;
            }
        }
        ox = nox;
        oy = noy;
        oz = noz;
        n_scat += scat ? 1u : 0u;
        n_wall += on_wall ? 1u : 0u;
        n_per += periodic ? 1u : 0u;
        // step VI and truncation
        const bool s_cap = n_scat >= scat_cap;
        const bool c_cap = col_cap && n_scat + n_wall >= max_col;
        if (absorbed || s_cap || c_cap || n_seg >= max_events) {
            fate = absorbed ? FATE_ABSORBED : s_cap ? FATE_MAX_SCATTER : c_cap ? FATE_MAX_COLLISIONS : FATE_MAX_EVENTS;
            alive = false;
            pending = true;
        }
    };

    unsigned long long next = first;
    const unsigned long long end = (unsigned long long)first + count;
    int cnt = 0;  // particles waiting in the warp's buffer (warp-uniform)
    for (;;) {
        const unsigned dead = __ballot_sync(FULL, !alive);
        if (dead && (__popc(dead) >= kRefill || next >= end || dead == FULL)) {
            if (pending) finish();
            const int need = __popc(dead);
            while (cnt < need && next < end) {
                // step I for the next 32 ids, whole warp
                const unsigned long long id = next + (unsigned long long)lane;
                const bool valid = id < end;
                const unsigned vmask = __ballot_sync(FULL, valid);
                if (valid) {
                    R ex, ey, ez, eox, eoy, eoz, et;
                    uint32_t mode, cy, cz;
                    int es;
                    if (!emit_particle<R, GEOM, SRC>(P, ctx, rk, alias_emit, (uint32_t)id, ex, ey, ez, eox, eoy, eoz,
                                                     et, mode, es, cy, cz))
                        flags |= FLAG_REJECTION_EXHAUSTED;
                    const int sl = cnt + __popc(vmask & lanemask_lt);
                    buf.x[sl] = ex;
                    buf.y[sl] = ey;
                    buf.z[sl] = ez;
                    buf.ox[sl] = eox;
                    buf.oy[sl] = eoy;
                    buf.oz[sl] = eoz;
                    buf.lam[sl] = __uint_as_float(fused[mode].z);
                    buf.pid[sl] = (uint32_t)id;
                    buf.sign[sl] = es;
                }
                cnt += __popc(vmask);
                next += 32ull;
                if (next > end) next = end;
                __syncwarp();
            }
            if (!alive) {
                const int rank = __popc(dead & lanemask_lt);
                if (rank < cnt) {
                    const int sl = cnt - 1 - rank;
                    x = buf.x[sl];
                    y = buf.y[sl];
                    z = buf.z[sl];
                    ox = buf.ox[sl];
                    oy = buf.oy[sl];
                    oz = buf.oz[sl];
                    lam = buf.lam[sl];
                    sign = buf.sign[sl];
                    pl = philox_lane(buf.pid[sl], inst, rk);
                    Lacc = 0;
                    n_seg = n_scat = n_wall = n_per = 0;
                    alive = true;
                }
            }
            cnt -= min(cnt, need);
            __syncwarp();
            if (!__any_sync(FULL, alive)) break;
        }
        if (alive) step(philox_flight(n_seg + 1u, pl, rk));
    }

    // warp totals into the slot's tallies, then the particle count
    double v0 = acc_sL.value(), v1 = acc_sL2.value();
    unsigned long long red[CNT_N] = {c_part, c_seg, c_scat, c_wall, c_per, c_trunc, c_abs};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(FULL, v0, o);
        v1 += __shfl_xor_sync(FULL, v1, o);
#pragma unroll
        for (int i = 0; i < CNT_N; ++i) red[i] += __shfl_xor_sync(FULL, red[i], o);
    }
    const uint32_t fl = __reduce_or_sync(FULL, flags);
    if (lane == 0) {
        atomicAdd(&T.sums[0], v0);
        atomicAdd(&T.sums[1], v1);
#pragma unroll
        for (int i = 0; i < CNT_N; ++i)
            if (red[i]) atomicAdd(&T.counters[i], red[i]);
        if (fl) atomicOr(&T.flags, fl);
        __threadfence();
        atomicAdd(&T.done, (unsigned long long)count);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) serve_kernel(const __grid_constant__ ServeArgs A)
{
    // per-warp copy of the slot being traced (parameters, round keys, table
    // pointers): the kernel outlives requests, so a slot's contents change
    // while it runs and are read afresh, through L2, for every item
    __shared__ ServeSlot s_slot[8];
    __shared__ ServeBuf s_buf[8];
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (blockDim.x > 256u || (blockDim.x & 31u) != 0u) {
        if (threadIdx.x == 0) atomicOr(A.status, FLAG_BAD_LAUNCH);
        return;
    }
    unsigned long long idle_since = global_ns();
    for (;;) {
        // lane 0 claims the next published item, or decides to leave
        int got = 0;
        uint32_t slot = 0, first = 0, count = 0;
        if (lane == 0) {
            got = -1;
            for (unsigned polls = 0; polls < kMaxPolls; ++polls) {
                if (load_acquire_sys(A.stop)) break;
                const unsigned long long tail = load_acquire_sys(A.tail);
                const unsigned long long h = *reinterpret_cast<volatile unsigned long long*>(A.head);
                if (h < tail) {
                    // read the item before claiming it: the host reuses a
                    // ring entry only after the head has passed it
                    const volatile ServeItem* it = A.items + (h & A.ring_mask);
                    const uint32_t s0 = it->slot, f0 = it->first, c0 = it->count;
                    if (atomicCAS(A.head, h, h + 1) == h) {
                        slot = s0;
                        first = f0;
                        count = c0;
                        got = 1;
                        break;
                    }
                    continue;  // another warp took it: try the next one at once
                }
                if (global_ns() - idle_since > A.idle_ns) break;
                __nanosleep(kSleepNs);
            }
        }
        // The host writes a slot and the tables it points to before it
        // publishes the slot's items; the tail was read with acquire
        // semantics at system scope, and this fence orders every later load
        // of the warp after it, so none of them is served from a line cached
        // before the host's writes (tables of retired requests may have
        // occupied the same addresses).
        if (lane == 0 && got > 0) __threadfence_system();
        got = __shfl_sync(FULL, got, 0);
        if (got < 0) break;
        slot = __shfl_sync(FULL, slot, 0);
        first = __shfl_sync(FULL, first, 0);
        count = __shfl_sync(FULL, count, 0);
        if (slot >= A.n_slots) {  // never published by the host; reported, skipped
            if (lane == 0) atomicOr(A.status, FLAG_BAD_LAUNCH);
            continue;
        }
        {
            static_assert(sizeof(ServeSlot) % 4 == 0, "slot copied in 32-bit words");
            const volatile uint32_t* src = reinterpret_cast<const volatile uint32_t*>(A.slots + slot);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_slot[warp]);
            for (int i = lane; i < (int)(sizeof(ServeSlot) / 4); i += 32) dst[i] = src[i];
        }
        __syncwarp();
        const ServeSlot& S = s_slot[warp];
        ServeTally& T = A.tallies[slot];
        switch (S.family) {
        case SERVE_SLAB: serve_item<LE_MC_GEOM_PLANES, LE_MC_SRC_WALLS>(S, T, s_buf[warp], first, count); break;
        case SERVE_FILM: serve_item<LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT>(S, T, s_buf[warp], first, count); break;
        case SERVE_POROUS: serve_item<LE_MC_GEOM_POROUS, LE_MC_SRC_GRADIENT>(S, T, s_buf[warp], first, count); break;
        default: serve_item<LE_MC_GEOM_BULK, LE_MC_SRC_GRADIENT>(S, T, s_buf[warp], first, count); break;
        }
        __syncwarp();
        idle_since = global_ns();
    }
}

}  // namespace

cudaError_t serve_occupancy(int threads, int* per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, serve_kernel, threads, 0);
}

cudaError_t launch_serve(const ServeArgs& a, int blocks, int threads, cudaStream_t st)
{
    serve_kernel<<<blocks, threads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lemc
