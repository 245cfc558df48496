// Request server: continuous batching of simulation requests on one GPU.
// A worker thread admits queued requests into slots (bounded by slot count
// and a device-memory budget).  An admitted request's parameters, Eq. 2 table
// and tallies stay in device memory until it retires; its particles are
// traced in epochs over consecutive particle-id ranges, each epoch published
// as work items to a ring that one resident persistent kernel
// (serve_kernel.cu) drains, so the particles of all admitted requests, of any
// geometry family and material, are interleaved inside that one kernel.  The
// worker polls the slots' particle counts and retires a request when its
// primary estimate reaches the target relative standard error or its budget
// is spent.  Declared in include/le_mc.h.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "le_mc_internal.h"
#include "le_mc_params.h"
#include "serve_kernel.h"

namespace lemc {
le_mc_status set_cuda_error(cudaError_t e, const char* where);
}  // namespace lemc

using namespace lemc;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    le_mc_material_desc mdesc{};
    std::vector<double> tab_v, tab_tau, tab_C;
    le_mc_geometry_desc gdesc{};
    le_mc_run_desc rdesc{};
    double target = 0.0;
    uint64_t budget = 0;
    int state = LE_MC_REQ_QUEUED;
    std::atomic<bool> cancel{false};
    std::atomic<int> epochs{0};
    double submit_s = 0, start_s = 0, done_s = 0, rel_err = 0;
    le_mc_tallies result{};
    // while active
    le_mc_material mat = nullptr;
    MaterialSums msums{};
    uint4* d_fused = nullptr;   // its Eq. 2 table on the device
    int slot = -1;
    bool inflight = false;      // an epoch is published and not yet complete
    uint64_t n_done = 0, n_next = 0;
    uint64_t to_publish = 0;    // particles of the current epoch not yet in the ring
    uint64_t item = 0;          // particles per work item of the current epoch
    double sums[2] = {0, 0};
    unsigned long long counters[CNT_N] = {};
    uint64_t footprint = 0;
};

// Family of the resident kernel that traces a request.
int family_of(const le_mc_geometry_desc& g, const le_mc_run_desc& r)
{
    if (g.kind == LE_MC_GEOM_PLANES) return r.source == LE_MC_SRC_WALLS ? SERVE_SLAB : SERVE_FILM;
    if (g.kind == LE_MC_GEOM_POROUS) return SERVE_POROUS;
    return SERVE_BULK;
}

// Relative standard error of the primary estimate (flux along the axis)
// from the accumulated per-particle sums; +inf until it is defined.
double rel_error(const Request& q)
{
    if (q.n_done < 2) return INFINITY;
    const double N = (double)q.n_done;
    const double mean = q.sums[0] / N;
    double var = (q.sums[1] - N * mean * mean) / (N - 1.0);
    if (var < 0.0) var = 0.0;
    if (mean == 0.0) return INFINITY;
    return sqrt(var / N) / fabs(mean);
}

// Particles for the next epoch: enough to reach the target if the current
// variance estimate holds (5 % margin), rounded up to 2^15, within budget.
uint64_t next_epoch(const Request& q, uint64_t pilot, uint64_t cap)
{
    const uint64_t left = q.budget - q.n_done;
    // the wish is formed and bounded in double: for a target far below the
    // error reached (the particles needed scale as the squared ratio) it can
    // exceed what a 64-bit integer holds, and a conversion of such a value,
    // or a rounding up that wraps, must not turn it into an empty epoch
    double want_d;
    if (q.n_done == 0) {
        want_d = (double)pilot;
    } else {
        const double re = rel_error(q);
        if (!isfinite(re)) {
            want_d = (double)q.n_done;
        } else {
            const double ratio = re / q.target;
            const double total = (double)q.n_done * ratio * ratio * 1.05;
            want_d = total > (double)q.n_done ? ceil(total - (double)q.n_done) : 1.0;
        }
    }
    const uint64_t lim = cap < left ? cap : left;
    if (!(want_d < (double)lim)) want_d = (double)lim;  // (also catches NaN)
    uint64_t want = want_d > 1.0 ? (uint64_t)want_d : 1;  // <= lim < 2^32
    const uint64_t quantum = 1ull << 15;
    want = (want + quantum - 1) / quantum * quantum;
    if (want > lim) want = lim;
    return want;
}

// Device memory an admitted request holds: the material's mode and alias
// tables, its Eq. 2 table for the resident kernel (the slot itself and its
// tallies are allocated with the server).
uint64_t footprint_of(int n_modes) { return (uint64_t)n_modes * (48 + 16) + 1024; }

// Particles per work item.  An item is what one warp traces before it claims
// again, so it bounds how long a new request's first items can wait: items
// hold about kItemSegments segments (~1 ms of a warp) by the request's own
// segments per particle (known after its pilot epoch; before that, 256
// particles or one item per warp, whichever is larger), and an epoch is cut
// into at least one item per warp so that even
// one request spreads over the GPU; never fewer than kItemMin particles (two
// per lane: a claim reads the ring in host memory) nor more than kItemMax.
constexpr double kItemSegments = 1.6e5;
constexpr uint64_t kItemMin = 64;
constexpr uint64_t kItemMax = 1ull << 14;
// Work items the ring holds (a power of two).
constexpr uint32_t kRingItems = 1u << 16;

}  // namespace

struct le_mc_server_s {
    le_mc_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_idle;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    std::vector<bool> slot_used;
    uint64_t next_id = 1;
    uint64_t hbm_in_use = 0;
    uint64_t submitted = 0, completed = 0, failed = 0, segments = 0, particles = 0;
    bool stopping = false;
    std::thread worker;

    // resident kernel state (worker thread only)
    cudaStream_t ks = nullptr, cs = nullptr;  // kernel stream, control stream (both non-blocking)
    cudaEvent_t ev_kernel = nullptr;          // recorded after each launch of the resident kernel
    bool launched = false;
    std::atomic<uint64_t> kernel_launches{0};
    unsigned char* d_block = nullptr;         // slots, tallies, head, status
    ServeSlot* d_slots = nullptr;
    ServeTally* d_tallies = nullptr;
    unsigned long long* d_head = nullptr;
    unsigned int* d_status = nullptr;
    unsigned char* h_ring = nullptr;          // mapped pinned: control block + items
    ServeControl* h_ctl = nullptr;
    ServeItem* h_items = nullptr;
    ServeArgs args{};
    ServeTally* h_tallies = nullptr;          // pinned read-back of the tallies (+ head)
    unsigned long long* h_head = nullptr;
    uint64_t tail = 0;                        // items published (host copy)
    uint64_t head_seen = 0;                   // items claimed, as of the last poll
    int blocks = 0, threads = 256;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void finish(Request* q, int state)
    {
        // caller holds mu; the request has no items left in the ring
        q->state = state;
        q->done_s = now();
        if (q->d_fused) cudaFreeAsync(q->d_fused, cs);
        q->d_fused = nullptr;
        if (q->mat) le_mc_destroy_material(q->mat);
        q->mat = nullptr;
        if (q->slot >= 0) slot_used[q->slot] = false;
        q->slot = -1;
        hbm_in_use -= q->footprint;
        if (state == LE_MC_REQ_DONE) ++completed; else ++failed;
    }

    cudaError_t setup_device();
    void teardown_device();
    le_mc_status admit(Request* q);
    bool kernel_running();
    cudaError_t ensure_kernel();
    bool publish_one(Request* q);
    void run();
};

cudaError_t le_mc_server_s::setup_device()
{
    const int n = cfg.max_slots;
    cudaError_t e = cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_kernel, cudaEventDisableTiming);
    const size_t b_slots = ((size_t)n * sizeof(ServeSlot) + 255) & ~(size_t)255;
    const size_t b_tal = ((size_t)n * sizeof(ServeTally) + 255) & ~(size_t)255;
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_block, b_slots + b_tal + 256);
    if (e == cudaSuccess) e = cudaMemset(d_block, 0, b_slots + b_tal + 256);
    if (e != cudaSuccess) return e;
    d_slots = reinterpret_cast<ServeSlot*>(d_block);
    d_tallies = reinterpret_cast<ServeTally*>(d_block + b_slots);
    d_head = reinterpret_cast<unsigned long long*>(d_block + b_slots + b_tal);
    d_status = reinterpret_cast<unsigned int*>(d_block + b_slots + b_tal + 8);
    const size_t b_ring = 256 + (size_t)kRingItems * sizeof(ServeItem);
    e = cudaHostAlloc((void**)&h_ring, b_ring, cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    memset(h_ring, 0, b_ring);
    h_ctl = reinterpret_cast<ServeControl*>(h_ring);
    h_items = reinterpret_cast<ServeItem*>(h_ring + 256);
    unsigned char* d_ring = nullptr;
    e = cudaHostGetDevicePointer((void**)&d_ring, h_ring, 0);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h_tallies, b_tal + 256);
    if (e != cudaSuccess) return e;
    h_head = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(h_tallies) + b_tal);
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = serve_occupancy(threads, &per_sm);
    if (e != cudaSuccess) return e;
    blocks = sms * (per_sm > 0 ? per_sm : 1);
    args.slots = d_slots;
    args.tallies = d_tallies;
    args.items = reinterpret_cast<const ServeItem*>(d_ring + 256);
    args.tail = reinterpret_cast<const unsigned long long*>(d_ring + offsetof(ServeControl, tail));
    args.stop = reinterpret_cast<const unsigned int*>(d_ring + offsetof(ServeControl, stop));
    args.head = d_head;
    args.status = d_status;
    args.ring_mask = kRingItems - 1u;
    args.n_slots = (uint32_t)n;
    args.idle_ns = (unsigned long long)(cfg.idle_exit_ms > 0 ? cfg.idle_exit_ms : 250) * 1000000ull;
    return cudaSuccess;
}

void le_mc_server_s::teardown_device()
{
    if (h_ctl) {
        __atomic_store_n(&h_ctl->stop, 1u, __ATOMIC_RELEASE);
        if (launched) cudaEventSynchronize(ev_kernel);
    }
    if (cs) cudaStreamSynchronize(cs);
    if (h_ring) cudaFreeHost(h_ring);
    if (h_tallies) cudaFreeHost(h_tallies);
    if (d_block) cudaFree(d_block);
    if (ev_kernel) cudaEventDestroy(ev_kernel);
    if (ks) cudaStreamDestroy(ks);
    if (cs) cudaStreamDestroy(cs);
}

bool le_mc_server_s::kernel_running()
{
    if (!launched) return false;
    const cudaError_t e = cudaEventQuery(ev_kernel);
    if (e == cudaErrorNotReady) return true;
    launched = false;
    return false;
}

// Launch the resident kernel unless it is still running (it leaves on its
// own after idle_exit_ms without work).
cudaError_t le_mc_server_s::ensure_kernel()
{
    if (kernel_running()) return cudaSuccess;
    cudaError_t e = launch_serve(args, blocks, threads, ks);
    if (e == cudaSuccess) e = cudaEventRecord(ev_kernel, ks);
    if (e == cudaSuccess) {
        launched = true;
        kernel_launches.fetch_add(1);
    }
    return e;
}

// Device state of a newly admitted request: material tables, its Eq. 2 table
// in the resident kernel's layout, its parameters in the slot, zero tallies.
le_mc_status le_mc_server_s::admit(Request* q)
{
    le_mc_status st = le_mc_create_material(&q->mdesc, &q->mat);
    if (st != LE_MC_OK) return st;
    MaterialView mv{};
    material_view(q->mat, &mv);
    q->msums = mv.sums;
    // Eq. 2 table: (threshold, alias, Lambda_j ln 2, Lambda_alias ln 2), the
    // same construction as the run kernels' shared-memory table
    const char* why = "";
    int n = 0;
    build_mode_table(&q->mdesc, nullptr, nullptr, nullptr, nullptr, 0, &n, &why);
    std::vector<double> om(n), v(n), tau(n), C(n), w(n);
    build_mode_table(&q->mdesc, om.data(), v.data(), tau.data(), C.data(), n, &n, &why);
    std::vector<uint32_t> thr(n), al(n);
    for (int i = 0; i < n; ++i) w[i] = C[i] / tau[i];
    if (build_alias(w.data(), n, thr.data(), al.data(), &why) != LE_MC_OK) return set_error(LE_MC_ERR_INVALID, "server", why);
    std::vector<uint4> fused(n);
    for (int i = 0; i < n; ++i) {
        const float lj = (float)(v[i] * tau[i]) * 0.693147180559945f;
        const float la = (float)(v[al[i]] * tau[al[i]]) * 0.693147180559945f;
        uint32_t bj, ba;
        memcpy(&bj, &lj, 4);
        memcpy(&ba, &la, 4);
        fused[i] = make_uint4(thr[i], al[i], bj, ba);
    }
    ServeSlot slot;
    memset(&slot, 0, sizeof(slot));
    KernelArgs a;
    memset(&a, 0, sizeof(a));
    TraceParams& P = a.p;
    fill_material(P, mv, true);
    fill_geometry(P, q->gdesc);
    le_mc_run_desc r = q->rdesc;
    fill_run(P, r);
    P.n_batch = 1;
    fill_consts(P);
    fill_round_keys(a);
    slot.p = P;
    slot.rk = a.rk;
    slot.family = family_of(q->gdesc, q->rdesc);
    cudaError_t e = cudaMallocAsync((void**)&q->d_fused, (size_t)n * sizeof(uint4), cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q->d_fused, fused.data(), (size_t)n * sizeof(uint4), cudaMemcpyHostToDevice, cs);
    slot.fused = q->d_fused;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_slots + q->slot, &slot, sizeof(slot), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_tallies + q->slot, 0, sizeof(ServeTally), cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);  // (the host struct and table are on this stack)
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_server: admission");
    return LE_MC_OK;
}

// Publish the next item of q's current epoch (items are written before the
// tail that exposes them; the caller then stores the tail).
bool le_mc_server_s::publish_one(Request* q)
{
    if (q->to_publish == 0 || tail - head_seen >= kRingItems) return false;
    const uint64_t first = q->n_done + q->n_next - q->to_publish;
    const uint64_t cnt = q->to_publish < q->item ? q->to_publish : q->item;
    ServeItem& it = h_items[tail & (kRingItems - 1u)];
    it.slot = (uint32_t)q->slot;
    it.first = (uint32_t)first;
    it.count = (uint32_t)cnt;
    it.pad = 0;
    ++tail;
    q->to_publish -= cnt;
    return true;
}

void le_mc_server_s::run()
{
    cudaSetDevice(device);
    const uint64_t pilot = cfg.pilot_particles;
    const uint64_t cap = cfg.max_epoch_particles;
    const size_t b_tal = (((size_t)cfg.max_slots * sizeof(ServeTally) + 255) & ~(size_t)255);
    double last_progress = now();
    for (;;) {
        std::vector<Request*> work, admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            // admission: free slot and device memory
            while (!queue.empty() && (int)active.size() < cfg.max_slots) {
                Request* q = queue.front();
                if (q->cancel) {
                    queue.pop_front();
                    q->done_s = now();
                    q->state = LE_MC_REQ_FAILED;
                    ++failed;
                    continue;
                }
                int n_modes = 0;
                const char* why = "";
                build_mode_table(&q->mdesc, nullptr, nullptr, nullptr, nullptr, 0, &n_modes, &why);
                const uint64_t fp = footprint_of(n_modes);
                if (!active.empty() && hbm_in_use + fp > cfg.hbm_budget_bytes) break;
                queue.pop_front();
                q->footprint = fp;
                hbm_in_use += fp;
                for (int i = 0; i < cfg.max_slots; ++i)
                    if (!slot_used[i]) { slot_used[i] = true; q->slot = i; break; }
                q->state = LE_MC_REQ_RUNNING;
                q->start_s = now();
                active.push_back(q);
                admitted.push_back(q);
            }
            if (active.empty()) {
                cv_idle.notify_all();
                if (stopping) return;
                cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
                continue;
            }
            work = active;
        }
        bool progressed = false;
        for (Request* q : admitted) {
            progressed = true;
            if (admit(q) != LE_MC_OK) {
                std::lock_guard<std::mutex> lk(mu);
                finish(q, LE_MC_REQ_FAILED);
                active.erase(std::find(active.begin(), active.end(), q));
            }
        }
        if (!admitted.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            work = active;
        }
        // read every slot's totals and the claimed-item count (one copy)
        bool any_inflight = false;
        for (Request* q : work) any_inflight = any_inflight || q->inflight;
        if (any_inflight) {
            cudaError_t e = cudaMemcpyAsync(h_tallies, d_tallies, b_tal + 8, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e == cudaSuccess) head_seen = *h_head;
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(mu);
                for (Request* q : work) finish(q, LE_MC_REQ_FAILED);
                active.clear();
                continue;
            }
        }
        bool reread = false;
        for (Request* q : work)
            if (q->inflight && h_tallies[q->slot].done >= q->n_done + q->n_next) reread = true;
        if (reread) {
            // the sums of a completed epoch are written before its count: a
            // second copy after seeing the count holds them in full
            cudaMemcpyAsync(h_tallies, d_tallies, b_tal, cudaMemcpyDeviceToHost, cs);
            cudaStreamSynchronize(cs);
        }
        for (Request* q : work) {
            if (q->slot < 0) continue;
            if (q->inflight) {
                // a cancelled request publishes nothing more: its epoch ends
                // with the items already in the ring
                if (q->cancel && q->to_publish > 0) {
                    q->n_next -= q->to_publish;
                    q->to_publish = 0;
                }
                const ServeTally& T = h_tallies[q->slot];
                if (T.done < q->n_done + q->n_next) continue;  // (its remaining items are published below)
                q->inflight = false;
                progressed = true;
                std::lock_guard<std::mutex> lk(mu);
                const uint64_t seg_before = q->counters[CNT_SEGMENTS], part_before = q->counters[CNT_PARTICLES];
                q->sums[0] = T.sums[0];
                q->sums[1] = T.sums[1];
                for (int i = 0; i < CNT_N; ++i) q->counters[i] = T.counters[i];
                q->n_done += q->n_next;
                q->n_next = 0;
                segments += q->counters[CNT_SEGMENTS] - seg_before;
                particles += q->counters[CNT_PARTICLES] - part_before;
                q->rel_err = rel_error(*q);
                le_mc_run_desc tot = q->rdesc;
                tot.n_particles = q->n_done;
                normalize(&q->gdesc, &tot, q->msums, q->sums, q->counters, &q->result);
                q->result.device_flags = T.flags;
                if (q->rel_err <= q->target || q->n_done >= q->budget || q->cancel) {
                    finish(q, q->cancel && q->rel_err > q->target ? LE_MC_REQ_FAILED : LE_MC_REQ_DONE);
                    active.erase(std::find(active.begin(), active.end(), q));
                    continue;
                }
            }
            if (!q->inflight) {
                if (q->cancel) {
                    std::lock_guard<std::mutex> lk(mu);
                    finish(q, LE_MC_REQ_FAILED);
                    active.erase(std::find(active.begin(), active.end(), q));
                    progressed = true;
                    continue;
                }
                // next epoch: its particle range goes to the ring
                q->n_next = next_epoch(*q, pilot, cap);
                q->to_publish = q->n_next;
                const uint64_t warps = (uint64_t)blocks * (threads / 32);
                const double spp = q->counters[CNT_PARTICLES] > 0
                                       ? (double)q->counters[CNT_SEGMENTS] / (double)q->counters[CNT_PARTICLES]
                                       : 0.0;
                // (before the pilot epoch has measured its segments per
                // particle: 256 particles, or one item per warp when the epoch
                // is larger than that, so a large first epoch is not cut
                // into tens of thousands of claims)
                uint64_t item = spp > 0.0 ? (uint64_t)(kItemSegments / spp)
                                          : std::max<uint64_t>(256, q->n_next / warps);
                item = std::min(item, std::max<uint64_t>(q->n_next / warps, 1));
                q->item = std::min(kItemMax, std::max(kItemMin, (item + 31) / 32 * 32));
                q->inflight = true;
                ++q->epochs;
                progressed = true;
            }
        }
        // Keep about half as many unclaimed items as the resident kernel has
        // warps in the ring, drawn round-robin, one item per request with
        // work per pass: the GPU stays busy with whatever work there is (one
        // large request alone fills it), and a new request's first items
        // wait behind a short queue rather than behind whole epochs of others.
        {
            const uint64_t warps = (uint64_t)blocks * (threads / 32);
            const uint64_t depth = std::max<uint64_t>(64, warps / 2);
            uint64_t unclaimed = tail - head_seen;
            bool more = true;
            const uint64_t tail0 = tail;
            while (more && unclaimed < depth) {
                more = false;
                for (Request* q : work) {
                    if (q->slot < 0 || !q->inflight || q->to_publish == 0) continue;
                    if (unclaimed >= depth) break;
                    if (publish_one(q)) {
                        ++unclaimed;
                        more = true;
                    }
                }
            }
            if (tail != tail0) __atomic_store_n(&h_ctl->tail, (unsigned long long)tail, __ATOMIC_RELEASE);
        }
        if (tail > head_seen) {
            const cudaError_t e = ensure_kernel();
            if (e != cudaSuccess) {
                set_cuda_error(e, "le_mc_server: resident kernel launch");
                std::lock_guard<std::mutex> lk(mu);
                for (Request* q : active) finish(q, LE_MC_REQ_FAILED);
                active.clear();
                continue;
            }
        }
        if (progressed) {
            last_progress = now();
        } else {
            // a server being destroyed gives its requests in flight a bounded
            // time to drain (a request whose items stopped making progress
            // would otherwise hold le_mc_server_destroy forever)
            bool stop_now;
            {
                std::lock_guard<std::mutex> lk(mu);
                stop_now = stopping && now() - last_progress > 60.0;
                if (stop_now) {
                    for (Request* q : active) {
                        // the kernel may still hold items of these requests:
                        // their tables are left allocated rather than freed
                        q->d_fused = nullptr;
                        q->mat = nullptr;
                        finish(q, LE_MC_REQ_FAILED);
                    }
                    active.clear();
                }
            }
            if (!stop_now) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
}

extern "C" {

le_mc_status le_mc_server_create(const le_mc_server_config* cfg, le_mc_server* out)
{
    if (!out) return set_error(LE_MC_ERR_INVALID, "le_mc_server_create", "out is null");
    *out = nullptr;
    le_mc_server_config c{};
    if (cfg) c = *cfg;
    if (c.max_slots == 0) c.max_slots = 8;
    if (c.max_slots < 1 || c.max_slots > 64) return set_error(LE_MC_ERR_INVALID, "le_mc_server_create", "max_slots out of 1..64");
    if (c.pilot_particles == 0) c.pilot_particles = 1ull << 16;
    if (c.max_epoch_particles == 0) c.max_epoch_particles = 1ull << 24;
    if (c.pilot_particles > 0xFFFFFFFFull || c.max_epoch_particles > 0xFFFFFFFFull)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_create", "epoch sizes must be < 2^32");
    std::unique_ptr<le_mc_server_s> s(new (std::nothrow) le_mc_server_s());
    if (!s) return set_error(LE_MC_ERR_NOMEM, "le_mc_server_create", "host allocation");
    cudaError_t e = cudaGetDevice(&s->device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_server_create");
    if (c.hbm_budget_bytes == 0) c.hbm_budget_bytes = free_b / 2;
    if (c.idle_exit_ms < 0 || c.idle_exit_ms > 60000)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_create", "idle_exit_ms out of 0..60000");
    s->cfg = c;
    s->slot_used.assign(c.max_slots, false);
    e = s->setup_device();
    if (e != cudaSuccess) {
        s->teardown_device();
        return set_cuda_error(e, "le_mc_server_create");
    }
    s->t0 = Clock::now();
    le_mc_server raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = raw;
    return LE_MC_OK;
}

le_mc_status le_mc_server_submit(le_mc_server s, const le_mc_material_desc* m, const le_mc_geometry_desc* g,
                                 const le_mc_run_desc* r, double target_rel_err, uint64_t* request_id)
{
    if (!s || !m || !g || !r || !request_id) return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", "null argument");
    const char* why = "";
    int n_modes = 0;
    if (build_mode_table(m, nullptr, nullptr, nullptr, nullptr, 0, &n_modes, &why) != LE_MC_OK)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", why);
    if (check_geometry(g, &why) != LE_MC_OK) return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", why);
    if (check_run(g, r, n_modes, &why) != LE_MC_OK) return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", why);
    if (r->source == LE_MC_SRC_PULSE || r->source == LE_MC_SRC_INITIAL || r->n_bins_x > 0 || r->n_hj > 0 || r->record_particles || r->first_particle ||
        r->map_ny > 0)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit",
                         "served requests are steady WALLS / GRADIENT runs without arrays");
    // what the resident kernel traces: FP32 trajectories, isotropic
    // relaxation events, black / diffuse / specular walls
    if (r->precision != LE_MC_PREC_FP32)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", "served requests use FP32 trajectories");
    if (m->scatter_g != 0.0)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", "served requests scatter isotropically");
    if (g->kind != LE_MC_GEOM_BULK && (g->wall_lo == LE_MC_WALL_PARTIAL || g->wall_hi == LE_MC_WALL_PARTIAL ||
                                       (g->kind == LE_MC_GEOM_POROUS && g->pore_wall == LE_MC_WALL_PARTIAL)))
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", "partially specular walls are not served");
    if (r->source == LE_MC_SRC_WALLS && g->kind != LE_MC_GEOM_PLANES)
        return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", "the walls source is served between planes only");
    if (!(target_rel_err > 0.0)) return set_error(LE_MC_ERR_INVALID, "le_mc_server_submit", "target_rel_err must be > 0");
    std::unique_ptr<Request> q(new (std::nothrow) Request());
    if (!q) return set_error(LE_MC_ERR_NOMEM, "le_mc_server_submit", "host allocation");
    q->mdesc = *m;
    if (m->kind == LE_MC_MAT_TABULATED) {
        q->tab_v.assign(m->tab_v, m->tab_v + m->n_modes);
        q->tab_tau.assign(m->tab_tau, m->tab_tau + m->n_modes);
        q->tab_C.assign(m->tab_C, m->tab_C + m->n_modes);
        q->mdesc.tab_v = q->tab_v.data();
        q->mdesc.tab_tau = q->tab_tau.data();
        q->mdesc.tab_C = q->tab_C.data();
    }
    q->gdesc = *g;
    q->rdesc = *r;
    q->target = target_rel_err;
    q->budget = r->n_particles;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return set_error(LE_MC_ERR_STATE, "le_mc_server_submit", "server is stopping");
    q->id = s->next_id++;
    q->submit_s = s->now();
    *request_id = q->id;
    s->queue.push_back(q.get());
    s->all[q->id] = std::move(q);
    ++s->submitted;
    s->cv_work.notify_one();
    return LE_MC_OK;
}

le_mc_status le_mc_server_poll(le_mc_server s, uint64_t id, le_mc_request_status* out)
{
    if (!s || !out) return set_error(LE_MC_ERR_INVALID, "le_mc_server_poll", "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return set_error(LE_MC_ERR_INVALID, "le_mc_server_poll", "unknown request id");
    const Request& q = *it->second;
    memset(out, 0, sizeof(*out));
    out->state = q.state;
    out->epochs = q.epochs;
    out->submit_s = q.submit_s;
    out->start_s = q.start_s;
    out->done_s = q.done_s;
    out->rel_err = q.rel_err;
    out->tallies = q.result;
    return LE_MC_OK;
}

le_mc_status le_mc_server_cancel(le_mc_server s, uint64_t id)
{
    if (!s) return set_error(LE_MC_ERR_INVALID, "le_mc_server_cancel", "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return set_error(LE_MC_ERR_INVALID, "le_mc_server_cancel", "unknown request id");
    it->second->cancel = true;
    s->cv_work.notify_one();
    return LE_MC_OK;
}

le_mc_status le_mc_server_wait_all(le_mc_server s, double timeout_s)
{
    if (!s) return set_error(LE_MC_ERR_INVALID, "le_mc_server_wait_all", "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->queue.empty() && s->active.empty(); });
    if (!ok) return set_error(LE_MC_ERR_TIMEOUT, "le_mc_server_wait_all", "requests still queued or running");
    return LE_MC_OK;
}

le_mc_status le_mc_server_stats(le_mc_server s, le_mc_server_counters* out)
{
    if (!s || !out) return set_error(LE_MC_ERR_INVALID, "le_mc_server_stats", "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->active = s->active.size();
    out->queued = s->queue.size();
    out->segments = s->segments;
    out->particles = s->particles;
    out->hbm_in_use = s->hbm_in_use;
    out->uptime_s = s->now();
    out->kernel_launches = s->kernel_launches.load();
    return LE_MC_OK;
}

le_mc_status le_mc_server_destroy(le_mc_server s)
{
    if (!s) return LE_MC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (Request* q : s->queue) q->cancel = true;
        for (Request* q : s->active) q->cancel = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    s->teardown_device();
    delete s;
    return LE_MC_OK;
}

}  // extern "C"
