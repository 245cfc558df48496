// Request server: continuous batching of simulation requests on one GPU.
// A worker thread admits queued requests into slots (bounded by slot count
// and a device-memory budget), traces each request in epochs with le_mc_run
// over consecutive particle-id ranges on the slot's own stream, polls the
// epochs without blocking, and retires a request when its primary estimate
// reaches the target relative standard error or its budget is spent.
// Declared in include/le_mc.h.
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

namespace lemc {
le_mc_status set_cuda_error(cudaError_t e, const char* where);
int run_ready(le_mc_run_handle h);
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
    le_mc_geometry geo = nullptr;
    MaterialSums msums{};
    le_mc_run_handle inflight = nullptr;
    int slot = -1;
    uint64_t n_done = 0, n_next = 0;
    double sums[2] = {0, 0};
    unsigned long long counters[CNT_N] = {};
    uint64_t footprint = 0;
};

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
    uint64_t want;
    if (q.n_done == 0) {
        want = pilot;
    } else {
        const double re = rel_error(q);
        if (!isfinite(re)) {
            want = q.n_done;
        } else {
            const double ratio = re / q.target;
            const double total = (double)q.n_done * ratio * ratio * 1.05;
            want = total > (double)q.n_done ? (uint64_t)ceil(total - (double)q.n_done) : 1;
        }
    }
    const uint64_t quantum = 1ull << 15;
    want = (want + quantum - 1) / quantum * quantum;
    if (want > cap) want = cap;
    if (want > left) want = left;
    return want;
}

uint64_t footprint_of(const Request& q, int n_modes, uint64_t cap)
{
    const uint64_t epoch = q.budget < cap ? q.budget : cap;
    // mode tables + one run allocation (header, long-first list and bitmap)
    return (uint64_t)n_modes * 48 + 4096 + epoch / 8 + (epoch < (1ull << 20) ? epoch : (1ull << 20)) * 4;
}

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
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_used;
    uint64_t next_id = 1;
    uint64_t hbm_in_use = 0;
    uint64_t submitted = 0, completed = 0, failed = 0, segments = 0, particles = 0;
    bool stopping = false;
    std::thread worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void finish(Request* q, int state)
    {
        // caller holds mu
        q->state = state;
        q->done_s = now();
        if (q->mat) le_mc_destroy_material(q->mat);
        if (q->geo) le_mc_destroy_geometry(q->geo);
        q->mat = nullptr;
        q->geo = nullptr;
        if (q->slot >= 0) slot_used[q->slot] = false;
        q->slot = -1;
        hbm_in_use -= q->footprint;
        if (state == LE_MC_REQ_DONE) ++completed; else ++failed;
    }

    void run();
};

void le_mc_server_s::run()
{
    cudaSetDevice(device);
    const uint64_t pilot = cfg.pilot_particles;
    const uint64_t cap = cfg.max_epoch_particles;
    for (;;) {
        std::vector<Request*> work;
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
                const uint64_t fp = footprint_of(*q, n_modes, cap);
                if (!active.empty() && hbm_in_use + fp > cfg.hbm_budget_bytes) break;
                queue.pop_front();
                q->footprint = fp;
                hbm_in_use += fp;
                for (int i = 0; i < cfg.max_slots; ++i)
                    if (!slot_used[i]) { slot_used[i] = true; q->slot = i; break; }
                q->state = LE_MC_REQ_RUNNING;
                q->start_s = now();
                active.push_back(q);
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
        for (Request* q : work) {
            // material and geometry on first use (outside the lock)
            if (!q->mat) {
                le_mc_status st = le_mc_create_material(&q->mdesc, &q->mat);
                if (st == LE_MC_OK) st = le_mc_create_geometry(&q->gdesc, &q->geo);
                MaterialView mv;
                if (st == LE_MC_OK && material_view(q->mat, &mv)) q->msums = mv.sums;
                if (st != LE_MC_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    finish(q, LE_MC_REQ_FAILED);
                    active.erase(std::find(active.begin(), active.end(), q));
                    progressed = true;
                    continue;
                }
            }
            if (q->inflight) {
                const int ready = run_ready(q->inflight);
                if (ready == 0) continue;
                le_mc_tallies t;
                const le_mc_status st = ready > 0 ? le_mc_read_tallies(q->inflight, &t) : LE_MC_ERR_STATE;
                le_mc_destroy_run(q->inflight);
                q->inflight = nullptr;
                progressed = true;
                std::lock_guard<std::mutex> lk(mu);
                if (st != LE_MC_OK) {
                    finish(q, LE_MC_REQ_FAILED);
                    active.erase(std::find(active.begin(), active.end(), q));
                    continue;
                }
                q->sums[0] += t.sum_sL;
                q->sums[1] += t.sum_sL2;
                q->counters[CNT_PARTICLES] += t.particles;
                q->counters[CNT_SEGMENTS] += t.segments;
                q->counters[CNT_SCATTERS] += t.scatters;
                q->counters[CNT_WALL] += t.wall_hits;
                q->counters[CNT_PERIODIC] += t.periodic;
                q->counters[CNT_TRUNCATED] += t.truncated;
                q->counters[CNT_ABSORBED] += t.absorbed;
                q->n_done += q->n_next;
                segments += t.segments;
                particles += t.particles;
                q->rel_err = rel_error(*q);
                le_mc_run_desc tot = q->rdesc;
                tot.n_particles = q->n_done;
                normalize(&q->gdesc, &tot, q->msums, q->sums, q->counters, &q->result);
                if (q->rel_err <= q->target || q->n_done >= q->budget || q->cancel) {
                    finish(q, q->cancel && q->rel_err > q->target ? LE_MC_REQ_FAILED : LE_MC_REQ_DONE);
                    active.erase(std::find(active.begin(), active.end(), q));
                    continue;
                }
            }
            // next epoch
            q->n_next = next_epoch(*q, pilot, cap);
            le_mc_run_desc r = q->rdesc;
            r.n_particles = q->n_next;
            r.first_particle = (uint32_t)q->n_done;
            le_mc_run_handle h = nullptr;
            const le_mc_status st = le_mc_run(q->mat, q->geo, &r, streams[q->slot], &h);
            ++q->epochs;
            progressed = true;
            if (st != LE_MC_OK) {
                if (h) le_mc_destroy_run(h);
                std::lock_guard<std::mutex> lk(mu);
                finish(q, LE_MC_REQ_FAILED);
                active.erase(std::find(active.begin(), active.end(), q));
                continue;
            }
            q->inflight = h;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
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
    s->cfg = c;
    s->streams.resize(c.max_slots, nullptr);
    s->slot_used.assign(c.max_slots, false);
    for (int i = 0; i < c.max_slots && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (cudaStream_t st : s->streams)
            if (st) cudaStreamDestroy(st);
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
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamDestroy(st);
    delete s;
    return LE_MC_OK;
}

}  // extern "C"
