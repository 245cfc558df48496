// Batches: many independent instances of one problem family traced by one
// persistent launch (queue positions run over the concatenated instances),
// optionally captured once as a CUDA graph and replayed, with a launch-shape
// autotuner.  Declared in include/le_mc.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "le_mc_internal.h"
#include "trace_kernel.cuh"
#include "le_mc_params.h"

namespace lemc {
cudaError_t batch_attr_f32(int src, bool diff, int threads, size_t smem, int* per_sm);
cudaError_t batch_attr_f64(int src, bool diff, int threads, size_t smem, int* per_sm);
cudaError_t batch_launch_f32(const KernelArgs& a, int src, bool diff, int blocks, int threads, size_t smem,
                             cudaStream_t st);
cudaError_t batch_launch_f64(const KernelArgs& a, int src, bool diff, int blocks, int threads, size_t smem,
                             cudaStream_t st);
cudaError_t launch_classify_f32(const KernelArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_classify_f64(const KernelArgs& a, int blocks, cudaStream_t st);
size_t batch_smem_f32(int src, int n_modes, int threads, int n_instances);
size_t batch_smem_f64(int src, int n_modes, int threads, int n_instances);
// material internals needed here (le_mc_api.cu)
le_mc_status set_cuda_error(cudaError_t e, const char* where);
}  // namespace lemc

using namespace lemc;

struct le_mc_batch_s {
    le_mc_material mat = nullptr;
    MaterialView mv{};
    int n = 0;
    std::vector<le_mc_geometry_desc> geoms;
    std::vector<le_mc_run_desc> runs;
    le_mc_geometry_desc geo0{};
    le_mc_run_desc run0{};
    int device = 0;
    int sms = 0;
    unsigned long long total = 0;   // particles in all instances
    // device memory: constant part (instances, offsets) and the part zeroed per launch
    unsigned char* dev = nullptr;
    size_t dev_bytes = 0, zero_off = 0, zero_bytes = 0;
    size_t off_inst = 0, off_offsets = 0, off_queue = 0, off_flags = 0, off_long_count = 0;
    size_t off_sums = 0, off_counters = 0, off_long_bits = 0, off_long_list = 0;
    uint32_t long_cap = 0, ext_cap = 0;
    le_mc_launch_config cfg{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    bool launched = false, failed = false, have_results = false;
    std::vector<double> sums;
    std::vector<unsigned long long> counters;
    unsigned int flags = 0;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void drop_graph(le_mc_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

bool fp32(const le_mc_batch b) { return b->run0.precision == LE_MC_PREC_FP32; }

// gradient-driven films whose walls are all diffuse use the specialised kernel
bool all_diffuse(const le_mc_batch b)
{
    return b->run0.source == LE_MC_SRC_GRADIENT && b->geo0.wall_lo == LE_MC_WALL_DIFFUSE &&
           b->geo0.wall_hi == LE_MC_WALL_DIFFUSE && b->mv.scatter_g == 0.0 && b->run0.n_hj <= 0;
}

// Kernel arguments for the whole batch.
KernelArgs make_args(le_mc_batch b)
{
    KernelArgs a;
    memset(&a, 0, sizeof(a));
    TraceParams& P = a.p;
    const le_mc_run_desc& r = b->run0;
    fill_material(P, b->mv, fp32(b));
    fill_geometry(P, b->geo0);
    fill_run(P, r);
    // (per-instance: thickness, drive, size and instance word come from the
    // instance table; the shared geometry is PLANES with diffuse pores unused)
    P.pore_wall = LE_MC_WALL_DIFFUSE;
    P.n_particles = 0;
    P.inst = 0;
    P.n_batch = 1;
    P.sums = nullptr;
    P.counters = nullptr;
    P.queue = reinterpret_cast<unsigned int*>(b->dev + b->off_queue);
    P.flags = reinterpret_cast<unsigned int*>(b->dev + b->off_flags);
    if (b->long_cap > 0) {
        P.long_list = reinterpret_cast<uint32_t*>(b->dev + b->off_long_list);
        P.long_bits = reinterpret_cast<uint32_t*>(b->dev + b->off_long_bits);
        P.long_count = reinterpret_cast<unsigned int*>(b->dev + b->off_long_count);
        P.long_cap = b->long_cap;
        P.ext_cap = b->ext_cap;
    }
    P.instances = reinterpret_cast<const BatchInstance*>(b->dev + b->off_inst);
    P.offsets = reinterpret_cast<const unsigned long long*>(b->dev + b->off_offsets);
    P.n_instances = b->n;
    P.refill_min = b->cfg.refill_min > 0 ? b->cfg.refill_min : 1;
    P.chunk = b->cfg.chunk > 0 ? b->cfg.chunk : 32;
    P.first = 0;
    P.inst_sums = reinterpret_cast<double*>(b->dev + b->off_sums);
    P.inst_counters = reinterpret_cast<unsigned long long*>(b->dev + b->off_counters);
    fill_consts(P);
    fill_round_keys(a);
    return a;
}

// Launch shape for the current config (sets the kernel's shared-memory attribute).
cudaError_t shape(le_mc_batch b, int* blocks, int* threads, size_t* smem)
{
    int t = b->cfg.threads_per_block > 0 ? b->cfg.threads_per_block : 512;
    const int src = b->run0.source;
    const size_t sm = fp32(b) ? batch_smem_f32(src, b->mv.n_modes, t, b->n) : batch_smem_f64(src, b->mv.n_modes, t, b->n);
    int per_sm = 0;
    const bool d = all_diffuse(b);
    cudaError_t e = fp32(b) ? batch_attr_f32(src, d, t, sm, &per_sm) : batch_attr_f64(src, d, t, sm, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (b->cfg.blocks_per_sm > 0 && b->cfg.blocks_per_sm < per_sm) per_sm = b->cfg.blocks_per_sm;
    *blocks = b->sms * per_sm;
    *threads = t;
    *smem = sm;
    return cudaSuccess;
}

// zero + classify + trace, enqueued on st (also the body of the graph)
cudaError_t enqueue(le_mc_batch b, cudaStream_t st, int blocks, int threads, size_t smem)
{
    const KernelArgs a = make_args(b);
    cudaError_t e = cudaMemsetAsync(b->dev + b->zero_off, 0, b->zero_bytes, st);
    if (e == cudaSuccess && b->long_cap > 0)
        e = fp32(b) ? launch_classify_f32(a, b->sms * 8, st) : launch_classify_f64(a, b->sms * 8, st);
    if (e == cudaSuccess)
        e = fp32(b) ? batch_launch_f32(a, b->run0.source, all_diffuse(b), blocks, threads, smem, st)
                    : batch_launch_f64(a, b->run0.source, all_diffuse(b), blocks, threads, smem, st);
    return e;
}

bool same_family(const le_mc_geometry_desc& g, const le_mc_geometry_desc& g0, const le_mc_run_desc& r,
                 const le_mc_run_desc& r0)
{
    return g.kind == g0.kind && g.wall_lo == g0.wall_lo && g.wall_hi == g0.wall_hi && g.spec_lo == g0.spec_lo &&
           g.spec_hi == g0.spec_hi && r.source == r0.source && r.precision == r0.precision && r.seed == r0.seed &&
           r.max_scatter == r0.max_scatter && r.max_events == r0.max_events &&
           r.max_collisions == r0.max_collisions;
}

}  // namespace

extern "C" {

le_mc_status le_mc_batch_create(le_mc_material m, int32_t n, const le_mc_geometry_desc* geoms,
                                const le_mc_run_desc* runs, le_mc_batch* out)
{
    if (!out) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "out is null");
    *out = nullptr;
    if (!m || !geoms || !runs || n < 1) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "null argument or n < 1");
    MaterialView mv{};
    if (!material_view(m, &mv)) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "bad material");
    const char* why = "";
    unsigned long long total = 0;
    for (int i = 0; i < n; ++i) {
        if (check_geometry(&geoms[i], &why) != LE_MC_OK) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", why);
        if (check_run(&geoms[i], &runs[i], mv.n_modes, &why) != LE_MC_OK)
            return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", why);
        if (geoms[i].kind != LE_MC_GEOM_PLANES)
            return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "batches take PLANES geometries");
        if (runs[i].source == LE_MC_SRC_PULSE || runs[i].source == LE_MC_SRC_INITIAL)
            return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "batches take WALLS or GRADIENT sources");
        if (runs[i].first_particle != 0)
            return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "batch instances start at particle 0");
        if (runs[i].n_bins_x > 0 || runs[i].n_hj > 0 || runs[i].n_samples > 0 || runs[i].record_particles ||
            runs[i].map_ny > 0)
            return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "profiles, maps, H_j, grids and records are not batched");
        if (!same_family(geoms[i], geoms[0], runs[i], runs[0]))
            return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create",
                             "instances must share walls, source kind, precision, seed and caps");
        total += runs[i].n_particles;
    }
    if (total > 0xFFFFFFFFull) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "more than 2^32 - 1 particles");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_batch_create");
    if (dev != mv.device) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_create", "material lives on another device");

    le_mc_batch b = new (std::nothrow) le_mc_batch_s();
    if (!b) return set_error(LE_MC_ERR_NOMEM, "le_mc_batch_create", "host allocation");
    b->mat = m;
    material_retain(m);
    b->mv = mv;
    b->n = n;
    b->geoms.assign(geoms, geoms + n);
    b->runs.assign(runs, runs + n);
    b->geo0 = geoms[0];
    b->run0 = runs[0];
    b->device = dev;
    b->total = total;
    b->cfg.threads_per_block = runs[0].threads_per_block;
    b->cfg.blocks_per_sm = runs[0].blocks_per_sm;
    b->cfg.refill_min = runs[0].refill_min;
    b->cfg.chunk = runs[0].chunk;
    b->cfg.use_graph = 0;
    b->long_cap = (uint32_t)(total < (1ull << 20) ? total : (1ull << 20));
    if (runs[0].schedule == 2 || total == 0) b->long_cap = 0;
    b->ext_cap = (b->long_cap > 0 && total <= kExtMaxParticles) ? (uint32_t)(total < kExtCap ? total : kExtCap) : 0;
    size_t off = 0;
    b->off_inst = off; off += (size_t)n * sizeof(BatchInstance);
    off = align_up(off, 256);
    b->off_offsets = off; off += (size_t)(n + 1) * sizeof(unsigned long long);
    off = align_up(off, 256);
    b->zero_off = off;
    b->off_queue = off; off += sizeof(unsigned long long);
    b->off_flags = off; off += sizeof(unsigned long long);
    b->off_long_count = off; off += 4 * sizeof(unsigned int);
    off = align_up(off, 256);
    b->off_sums = off; off += (size_t)n * 2 * sizeof(double);
    off = align_up(off, 256);
    b->off_counters = off; off += (size_t)n * CNT_N * sizeof(unsigned long long);
    off = align_up(off, 256);
    if (b->long_cap > 0) {
        b->off_long_bits = off; off += (size_t)((total + 31) / 32) * sizeof(uint32_t);
        off = align_up(off, 256);
    }
    b->zero_bytes = off - b->zero_off;
    if (b->long_cap > 0) {
        b->off_long_list = off; off += (size_t)(b->ext_cap + b->long_cap) * sizeof(uint32_t);
    }
    b->dev_bytes = align_up(off, 256);
    std::vector<BatchInstance> inst(n);
    std::vector<unsigned long long> offsets(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        inst[i].L = geoms[i].L;
        inst[i].dT_lo = runs[i].dT_lo;
        inst[i].dT_hi = runs[i].dT_hi;
        inst[i].dTdz = runs[i].dTdz;
        inst[i].lam_cut = runs[i].long_mfp_cut > 0.0 ? runs[i].long_mfp_cut : 32.0 * geoms[i].L;
        inst[i].inst_id = runs[i].instance_id;
        inst[i].n_particles = (uint32_t)runs[i].n_particles;
        fill_instance32(inst[i]);
        offsets[i + 1] = offsets[i] + runs[i].n_particles;
    }
    b->sums.assign((size_t)n * 2, 0.0);
    b->counters.assign((size_t)n * CNT_N, 0ull);
    e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = alloc_fault_injected() ? cudaErrorMemoryAllocation : cudaMalloc((void**)&b->dev, b->dev_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(b->dev + b->off_inst, inst.data(), n * sizeof(BatchInstance), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->dev + b->off_offsets, offsets.data(), (n + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev_stop);
    if (e != cudaSuccess) {
        le_mc_batch_destroy(b);
        return set_cuda_error(e, "le_mc_batch_create");
    }
    *out = b;
    return LE_MC_OK;
}

le_mc_status le_mc_batch_set_config(le_mc_batch b, const le_mc_launch_config* cfg)
{
    if (!b || !cfg) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_set_config", "null argument");
    if (cfg->threads_per_block < 0 || cfg->threads_per_block > 512 || cfg->threads_per_block % 32 != 0 ||
        cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32 || cfg->refill_min < 0 || cfg->refill_min > 32 ||
        cfg->chunk < 0 || cfg->chunk % 32 != 0 || cfg->chunk > (1 << 20))
        return set_error(LE_MC_ERR_INVALID, "le_mc_batch_set_config", "launch shape out of range");
    b->cfg = *cfg;
    drop_graph(b);
    return LE_MC_OK;
}

le_mc_status le_mc_batch_launch(le_mc_batch b, void* stream)
{
    if (!b) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_launch", "null batch");
    if (b->failed) return set_error(LE_MC_ERR_STATE, "le_mc_batch_launch", "batch failed earlier");
    cudaStream_t st = (cudaStream_t)stream;
    int blocks = 0, threads = 0;
    size_t smem = 0;
    cudaError_t e = shape(b, &blocks, &threads, &smem);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_start, st);
    if (e == cudaSuccess) {
        if (b->cfg.use_graph) {
            if (!b->exec) {
                // capture once on a private stream (the caller's may be the
                // legacy default stream, which cannot be captured); the graph
                // is then replayed on the caller's stream
                if (!b->graph_stream) e = cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaStreamBeginCapture(b->graph_stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const cudaError_t e2 = enqueue(b, b->graph_stream, blocks, threads, smem);
                    e = cudaStreamEndCapture(b->graph_stream, &b->graph);
                    if (e2 != cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, st);
        } else {
            e = enqueue(b, st, blocks, threads, smem);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_stop, st);
    if (e != cudaSuccess) {
        b->failed = true;
        drop_graph(b);
        return set_cuda_error(e, "le_mc_batch_launch");
    }
    b->launched = true;
    b->have_results = false;
    return LE_MC_OK;
}

le_mc_status le_mc_batch_wait(le_mc_batch b)
{
    if (!b) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_wait", "null batch");
    if (b->failed) return set_error(LE_MC_ERR_STATE, "le_mc_batch_wait", "batch failed earlier");
    if (!b->launched) return set_error(LE_MC_ERR_STATE, "le_mc_batch_wait", "nothing launched");
    const cudaError_t e = cudaEventSynchronize(b->ev_stop);
    if (e != cudaSuccess) {
        b->failed = true;
        return set_cuda_error(e, "le_mc_batch_wait");
    }
    return LE_MC_OK;
}

le_mc_status le_mc_batch_read(le_mc_batch b, int32_t i, le_mc_tallies* out)
{
    if (!b || !out || i < 0 || i >= b->n) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_read", "bad argument");
    if (!b->have_results) {
        le_mc_status s = le_mc_batch_wait(b);
        if (s != LE_MC_OK) return s;
        cudaError_t e = cudaMemcpy(b->sums.data(), b->dev + b->off_sums, b->sums.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->counters.data(), b->dev + b->off_counters,
                           b->counters.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&b->flags, b->dev + b->off_flags, sizeof(unsigned int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            b->failed = true;
            return set_cuda_error(e, "le_mc_batch_read");
        }
        b->have_results = true;
    }
    memset(out, 0, sizeof(*out));
    normalize(&b->geoms[i], &b->runs[i], b->mv.sums, &b->sums[2 * (size_t)i], &b->counters[(size_t)CNT_N * i], out);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, b->ev_start, b->ev_stop);
    out->kernel_ms = ms;
    out->kernel_launches = b->long_cap > 0 ? 2 : 1;
    out->device_flags = b->flags;
    return LE_MC_OK;
}

le_mc_status le_mc_batch_autotune(le_mc_batch b, void* stream, const char* cache_path, le_mc_launch_config* best)
{
    if (!b || !best) return set_error(LE_MC_ERR_INVALID, "le_mc_batch_autotune", "null argument");
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, b->device);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_batch_autotune");
    char key[512];
    snprintf(key, sizeof(key), "geom=%d walls=%d,%d src=%d prec=%d modes=%d gpu=%s", b->geo0.kind, b->geo0.wall_lo,
             b->geo0.wall_hi, b->run0.source, b->run0.precision, b->mv.n_modes, prop.name);
    for (char* c = key; *c; ++c)
        if (*c == '\n' || *c == '|') *c = ' ';
    const int use_graph = b->cfg.use_graph;
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                char* bar = strchr(line, '|');
                if (!bar) continue;
                *bar = '\0';
                if (strcmp(line, key) != 0) continue;
                le_mc_launch_config c{};
                if (sscanf(bar + 1, "%d %d %d %d %f", &c.threads_per_block, &c.blocks_per_sm, &c.refill_min, &c.chunk,
                           &c.ms) == 5) {
                    c.use_graph = use_graph;
                    fclose(f);
                    *best = c;
                    return le_mc_batch_set_config(b, &c);
                }
            }
            fclose(f);
        }
    }
    const int threads[] = {128, 256, 512};
    const int refills[] = {1, 4};
    const int chunks[] = {32, 256};
    le_mc_launch_config top{};
    top.ms = 3.0e38f;
    for (int t : threads)
        for (int rf : refills)
            for (int ch : chunks) {
                le_mc_launch_config c{};
                c.threads_per_block = t;
                c.blocks_per_sm = 0;
                c.refill_min = rf;
                c.chunk = ch;
                c.use_graph = 0;
                le_mc_status s = le_mc_batch_set_config(b, &c);
                if (s != LE_MC_OK) return s;
                float ms = 0.0f;
                for (int rep = 0; rep < 2; ++rep) {  // warm-up, then timed
                    s = le_mc_batch_launch(b, stream);
                    if (s != LE_MC_OK) return s;
                    s = le_mc_batch_wait(b);
                    if (s != LE_MC_OK) return s;
                    cudaEventElapsedTime(&ms, b->ev_start, b->ev_stop);
                }
                if (ms < top.ms) {
                    top = c;
                    top.ms = ms;
                }
            }
    top.use_graph = use_graph;
    le_mc_status s = le_mc_batch_set_config(b, &top);
    if (s != LE_MC_OK) return s;
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s|%d %d %d %d %.4f\n", key, top.threads_per_block, top.blocks_per_sm, top.refill_min, top.chunk,
                    top.ms);
            fclose(f);
        }
    }
    *best = top;
    return LE_MC_OK;
}

le_mc_status le_mc_batch_destroy(le_mc_batch b)
{
    if (!b) return LE_MC_OK;
    // launches in flight read the material tables: let them finish first
    if (b->launched && !b->failed) cudaEventSynchronize(b->ev_stop);
    drop_graph(b);
    if (b->dev) cudaFree(b->dev);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_stop) cudaEventDestroy(b->ev_stop);
    if (b->graph_stream) cudaStreamDestroy(b->graph_stream);
    material_drop(b->mat);
    delete b;
    return LE_MC_OK;
}

}  // extern "C"
