// C ABI of the le_mc library (declared in include/le_mc.h): handle
// lifetimes, device memory, launches, read-back and normalisation.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "le_mc_internal.h"
#include "trace_kernel.cuh"
#include "le_mc_params.h"

namespace lemc {
cudaError_t launch_trace_f32(const KernelArgs& a, int geom, int src, bool profile, int blocks, int threads,
                             size_t smem, cudaStream_t st);
cudaError_t launch_trace_f64(const KernelArgs& a, int geom, int src, bool profile, int blocks, int threads,
                             size_t smem, cudaStream_t st);
cudaError_t occupancy_trace_f32(int geom, int src, bool profile, int threads, size_t smem, int* per_sm);
cudaError_t occupancy_trace_f64(int geom, int src, bool profile, int threads, size_t smem, int* per_sm);
cudaError_t occupancy_trace_for_f32(const TraceParams& p, bool profile, int threads, size_t smem, int* per_sm);
cudaError_t occupancy_trace_for_f64(const TraceParams& p, bool profile, int threads, size_t smem, int* per_sm);
cudaError_t smem_trace_f32(int geom, int src, bool profile, int n_modes, int threads, int prof_len, int hj_len,
                           size_t* bytes);
cudaError_t smem_trace_f64(int geom, int src, bool profile, int n_modes, int threads, int prof_len, int hj_len,
                           size_t* bytes);
cudaError_t launch_classify_f32(const KernelArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_classify_f64(const KernelArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, size_t n, cudaStream_t st);
cudaError_t launch_sample_modes(const uint2* table, int n_modes, const uint32_t* words, int32_t* out, size_t n,
                                cudaStream_t st);
}  // namespace lemc

using namespace lemc;

namespace {

thread_local char g_err[512] = "";

le_mc_status fail(le_mc_status s, const char* fmt, const char* detail = nullptr)
{
    if (detail) snprintf(g_err, sizeof(g_err), "%s: %s", fmt, detail);
    else snprintf(g_err, sizeof(g_err), "%s", fmt);
    return s;
}

// Device allocations of materials and runs, through the failure-test hook.
static cudaError_t alloc_async(void** p, size_t bytes, cudaStream_t s)
{
    if (alloc_fault_injected()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, s);
}

le_mc_status cuda_fail(cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) return fail(LE_MC_ERR_NOMEM, where, cudaGetErrorString(e));
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return fail(LE_MC_ERR_NODEV, where, cudaGetErrorString(e));
    return fail(LE_MC_ERR_CUDA, where, cudaGetErrorString(e));
}

#define CUDA_TRY(call, where)                               \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

}  // namespace

struct le_mc_material_s {
    std::atomic<int> refs{1};
    le_mc_material_desc desc{};
    int n_modes = 0;
    int device = 0;
    MaterialSums sums{};
    std::vector<double> omega, v, tau, C;
    void* d_props32 = nullptr;   // float2[n]
    void* d_props64 = nullptr;   // double2[n]
    uint2* d_alias_scat = nullptr;
    uint2* d_alias_emit = nullptr;
    uint2* d_alias_init = nullptr;
    // set once le_mc_run_noalloc has launched work reading these tables: such
    // work holds no reference, so releasing the tables waits for the device
    std::atomic<bool> noalloc_used{false};
};

struct le_mc_geometry_s {
    std::atomic<int> refs{1};
    le_mc_geometry_desc desc{};
};

struct le_mc_run_s {
    le_mc_material mat = nullptr;
    le_mc_geometry geo = nullptr;
    le_mc_run_desc desc{};
    cudaStream_t stream = nullptr;
    int device = 0;
    unsigned char* dev = nullptr;  // one stream-ordered allocation
    size_t dev_bytes = 0;
    size_t off_sums = 0, off_counters = 0, off_queue = 0, off_flags = 0;
    size_t off_prof = 0, off_hj = 0, off_grid = 0, off_records = 0;
    size_t off_long_list = 0, off_long_bits = 0, off_long_count = 0;
    uint32_t long_cap = 0, ext_cap = 0;
    size_t prof_len = 0, hj_len = 0, grid_len = 0;
    cudaEvent_t ev_start = nullptr, ev_mid = nullptr, ev_stop = nullptr;
    bool failed = false;
    bool have_header = false;
    double sums[2] = {0, 0};
    unsigned long long counters[CNT_N] = {};
    unsigned int flags = 0;
    uint32_t launches = 0;
    uint32_t long_listed = 0, extreme_traced = 0;
};

namespace {

void material_release(le_mc_material m)
{
    if (!m) return;
    if (m->refs.fetch_sub(1) != 1) return;
    // Every run and batch that used the tables has finished (they hold a
    // reference until destroyed, and destroying them waits for their device
    // work), so the stream-ordered frees need no device-wide synchronisation.
    // le_mc_run_noalloc holds no reference (it may not allocate one), and its
    // kernels may still be reading the tables on a stream the legacy stream
    // does not order against, so a material it has used waits for the whole
    // device first.
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    if (m->noalloc_used.load()) cudaDeviceSynchronize();
    if (m->d_props32) cudaFreeAsync(m->d_props32, 0);
    if (m->d_props64) cudaFreeAsync(m->d_props64, 0);
    if (m->d_alias_scat) cudaFreeAsync(m->d_alias_scat, 0);
    if (m->d_alias_emit) cudaFreeAsync(m->d_alias_emit, 0);
    if (m->d_alias_init) cudaFreeAsync(m->d_alias_init, 0);
    cudaSetDevice(cur);
    delete m;
}

void geometry_release(le_mc_geometry g)
{
    if (!g) return;
    if (g->refs.fetch_sub(1) != 1) return;
    delete g;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace lemc {
// Internal access for the batch and static-scratch translation units.

bool material_view(le_mc_material m, MaterialView* out)
{
    if (!m) return false;
    out->props32 = m->d_props32;
    out->props64 = m->d_props64;
    out->alias_scat = m->d_alias_scat;
    out->alias_emit = m->d_alias_emit;
    out->alias_init = m->d_alias_init;
    out->n_modes = m->n_modes;
    out->device = m->device;
    out->sums = m->sums;
    out->scatter_g = m->desc.scatter_g;
    return true;
}

bool geometry_view(le_mc_geometry g, le_mc_geometry_desc* out)
{
    if (!g) return false;
    *out = g->desc;
    return true;
}

void material_mark_noalloc(le_mc_material m)
{
    if (m) m->noalloc_used.store(true);
}

void material_retain(le_mc_material m)
{
    if (m) m->refs.fetch_add(1);
}

void material_drop(le_mc_material m) { material_release(m); }

le_mc_status set_error(le_mc_status s, const char* what, const char* detail) { return fail(s, what, detail); }

le_mc_status set_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }

// 1 when the run's device work is complete, 0 while it runs, -1 on error.
int run_ready(le_mc_run_handle h)
{
    if (!h || h->failed) return -1;
    if (!h->launches) return 1;
    const cudaError_t e = cudaEventQuery(h->ev_stop);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    h->failed = true;
    return -1;
}
}  // namespace lemc

extern "C" {

const char* le_mc_last_error(void) { return g_err; }
int32_t le_mc_abi_version(void) { return LE_MC_ABI_VERSION; }

int32_t le_mc_struct_size(int32_t which)
{
    switch (which) {
    case 0: return (int32_t)sizeof(le_mc_material_desc);
    case 1: return (int32_t)sizeof(le_mc_geometry_desc);
    case 2: return (int32_t)sizeof(le_mc_run_desc);
    case 3: return (int32_t)sizeof(le_mc_tallies);
    case 4: return (int32_t)sizeof(le_mc_particle);
    case 5: return (int32_t)sizeof(le_mc_launch_config);
    default: return -1;
    }
}

le_mc_status le_mc_material_table(const le_mc_material_desc* desc, double* omega, double* v, double* tau,
                                  double* C, int32_t capacity, int32_t* n_modes)
{
    const char* why = "";
    int n = 0;
    if (!n_modes) return fail(LE_MC_ERR_INVALID, "n_modes output is null");
    const int st = build_mode_table(desc, nullptr, nullptr, nullptr, nullptr, 0, &n, &why);
    if (st != LE_MC_OK) return fail((le_mc_status)st, "le_mc_material_table", why);
    *n_modes = n;
    if (omega && v && tau && C) {
        if (capacity < n) return fail(LE_MC_ERR_INVALID, "le_mc_material_table: capacity too small");
        build_mode_table(desc, omega, v, tau, C, capacity, &n, &why);
    }
    return LE_MC_OK;
}

le_mc_status le_mc_alias_table(const double* weights, int32_t n, uint32_t* threshold, uint32_t* alias)
{
    const char* why = "";
    if (!weights || !threshold || !alias) return fail(LE_MC_ERR_INVALID, "le_mc_alias_table: null pointer");
    const int st = build_alias(weights, n, threshold, alias, &why);
    if (st != LE_MC_OK) return fail((le_mc_status)st, "le_mc_alias_table", why);
    return LE_MC_OK;
}

le_mc_status le_mc_test_fail_allocation(int32_t after)
{
    set_alloc_fault(after);
    return LE_MC_OK;
}

le_mc_status le_mc_map_solid(const le_mc_geometry_desc* g, int32_t map_ny, int32_t map_nz, double* fraction)
{
    const char* why = nullptr;
    if (!g || !fraction) return fail(LE_MC_ERR_INVALID, "le_mc_map_solid: null pointer");
    if (check_geometry(g, &why) != LE_MC_OK) return fail(LE_MC_ERR_INVALID, "le_mc_map_solid", why);
    if (g->kind != LE_MC_GEOM_POROUS) return fail(LE_MC_ERR_INVALID, "le_mc_map_solid: needs the POROUS geometry");
    if (map_ny < 1 || map_nz < 1 || map_ny > LE_MC_MAX_MAP || map_nz > LE_MC_MAX_MAP)
        return fail(LE_MC_ERR_INVALID, "le_mc_map_solid: map_ny, map_nz out of 1..LE_MC_MAX_MAP");
    map_solid_fractions(g->pitch, g->radius, map_ny, map_nz, fraction);
    return LE_MC_OK;
}

le_mc_status le_mc_truncation_study(const double* H, const double* H_se, int32_t n, double resolved, int32_t first,
                                    le_mc_truncation* out)
{
    const char* why = "";
    if (truncation_study(H, H_se, n, resolved, first, out, &why) != LE_MC_OK)
        return fail(LE_MC_ERR_INVALID, "le_mc_truncation_study", why);
    return LE_MC_OK;
}

le_mc_status le_mc_truncation_tail(const le_mc_truncation* study, int32_t K, double* dropped)
{
    if (!study || !dropped) return fail(LE_MC_ERR_INVALID, "le_mc_truncation_tail: null pointer");
    if (K < 0) return fail(LE_MC_ERR_INVALID, "le_mc_truncation_tail: K must be >= 0");
    *dropped = truncation_tail(study, K);
    return LE_MC_OK;
}

le_mc_status le_mc_create_material(const le_mc_material_desc* desc, le_mc_material* out)
{
    if (!out) return fail(LE_MC_ERR_INVALID, "le_mc_create_material: out is null");
    *out = nullptr;
    const char* why = "";
    int n = 0;
    int st = build_mode_table(desc, nullptr, nullptr, nullptr, nullptr, 0, &n, &why);
    if (st != LE_MC_OK) return fail((le_mc_status)st, "le_mc_create_material", why);
    le_mc_material m = new (std::nothrow) le_mc_material_s();
    if (!m) return fail(LE_MC_ERR_NOMEM, "le_mc_create_material: host allocation");
    m->desc = *desc;
    m->desc.tab_v = m->desc.tab_tau = m->desc.tab_C = nullptr;
    m->n_modes = n;
    m->omega.resize(n); m->v.resize(n); m->tau.resize(n); m->C.resize(n);
    build_mode_table(desc, m->omega.data(), m->v.data(), m->tau.data(), m->C.data(), n, &n, &why);
    std::vector<double> w_emit(n), w_scat(n);
    std::vector<float> props32(2 * (size_t)n);
    std::vector<double> props64(2 * (size_t)n);
    m->sums.C_tot = 0.0;
    m->sums.Cv_sum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double lam = m->v[i] * m->tau[i];
        w_emit[i] = m->C[i] * m->v[i];  // boundary / gradient / pulse emission
        w_scat[i] = m->C[i] / m->tau[i];  // normalised Eq. 2
        m->sums.C_tot += m->C[i];
        m->sums.Cv_sum += w_emit[i];
        props64[2 * i] = lam;
        props64[2 * i + 1] = m->v[i];
        props32[2 * i] = (float)lam;
        props32[2 * i + 1] = (float)m->v[i];
    }
    std::vector<uint32_t> thr_e(n), al_e(n), thr_s(n), al_s(n), thr_i(n), al_i(n);
    st = build_alias(w_emit.data(), n, thr_e.data(), al_e.data(), &why);
    if (st == LE_MC_OK) st = build_alias(w_scat.data(), n, thr_s.data(), al_s.data(), &why);
    if (st == LE_MC_OK) st = build_alias(m->C.data(), n, thr_i.data(), al_i.data(), &why);  // initial condition
    if (st != LE_MC_OK) { delete m; return fail((le_mc_status)st, "le_mc_create_material", why); }
    std::vector<uint2> ae(n), as(n), ai(n);
    for (int i = 0; i < n; ++i) {
        ae[i] = make_uint2(thr_e[i], al_e[i]);
        as[i] = make_uint2(thr_s[i], al_s[i]);
        ai[i] = make_uint2(thr_i[i], al_i[i]);
    }
    // stream-ordered pool on the legacy stream, complete before returning
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = alloc_async(&m->d_props32, props32.size() * sizeof(float), 0);
    if (e == cudaSuccess) e = alloc_async(&m->d_props64, props64.size() * sizeof(double), 0);
    if (e == cudaSuccess) e = alloc_async((void**)&m->d_alias_scat, n * sizeof(uint2), 0);
    if (e == cudaSuccess) e = alloc_async((void**)&m->d_alias_emit, n * sizeof(uint2), 0);
    if (e == cudaSuccess) e = alloc_async((void**)&m->d_alias_init, n * sizeof(uint2), 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_props32, props32.data(), props32.size() * sizeof(float), cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_props64, props64.data(), props64.size() * sizeof(double), cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_alias_scat, as.data(), n * sizeof(uint2), cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_alias_emit, ae.data(), n * sizeof(uint2), cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_alias_init, ai.data(), n * sizeof(uint2), cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        material_release(m);
        return cuda_fail(e, "le_mc_create_material");
    }
    *out = m;
    return LE_MC_OK;
}

le_mc_status le_mc_destroy_material(le_mc_material m)
{
    material_release(m);
    return LE_MC_OK;
}

le_mc_status le_mc_create_geometry(const le_mc_geometry_desc* desc, le_mc_geometry* out)
{
    if (!out) return fail(LE_MC_ERR_INVALID, "le_mc_create_geometry: out is null");
    *out = nullptr;
    const char* why = "";
    const int st = check_geometry(desc, &why);
    if (st != LE_MC_OK) return fail((le_mc_status)st, "le_mc_create_geometry", why);
    le_mc_geometry g = new (std::nothrow) le_mc_geometry_s();
    if (!g) return fail(LE_MC_ERR_NOMEM, "le_mc_create_geometry: host allocation");
    g->desc = *desc;
    *out = g;
    return LE_MC_OK;
}

le_mc_status le_mc_destroy_geometry(le_mc_geometry g)
{
    geometry_release(g);
    return LE_MC_OK;
}

le_mc_status le_mc_run(le_mc_material m, le_mc_geometry g, const le_mc_run_desc* desc, void* stream,
                       le_mc_run_handle* out)
{
    if (!out) return fail(LE_MC_ERR_INVALID, "le_mc_run: out is null");
    *out = nullptr;
    if (!m || !g || !desc) return fail(LE_MC_ERR_INVALID, "le_mc_run: null handle or descriptor");
    const char* why = "";
    int st = check_run(&g->desc, desc, m->n_modes, &why);
    if (st != LE_MC_OK) return fail((le_mc_status)st, "le_mc_run", why);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "le_mc_run: cudaGetDevice");
    if (dev != m->device) return fail(LE_MC_ERR_INVALID, "le_mc_run: material lives on another device");

    le_mc_run_handle h = new (std::nothrow) le_mc_run_s();
    if (!h) return fail(LE_MC_ERR_NOMEM, "le_mc_run: host allocation");
    h->desc = *desc;
    h->stream = (cudaStream_t)stream;
    h->device = dev;
    const le_mc_run_desc& r = h->desc;
    // the PROFILE kernels tally slab profiles (PLANES) or steady maps (POROUS)
    const bool has_map = r.map_ny > 0 && r.map_nz > 0;
    const bool profile = r.n_bins_x > 0 || has_map;
    h->prof_len = has_map ? (size_t)2 * r.n_batch * r.map_ny * r.map_nz
                : profile ? (size_t)4 * r.n_batch * (r.n_bins_x + 1) : 0;
    h->hj_len = (size_t)2 * r.n_hj;
    h->grid_len = r.n_samples > 0 ? (size_t)r.n_samples * r.grid_nx * r.grid_ny * r.grid_nz : 0;
    size_t off = 0;
    h->off_sums = off; off += 2 * sizeof(double);
    h->off_counters = off; off += CNT_N * sizeof(unsigned long long);
    h->off_queue = off; off += sizeof(unsigned long long);
    h->off_flags = off; off += sizeof(unsigned long long);
    off = align_up(off, 256);
    h->off_prof = off; off += h->prof_len * sizeof(double);
    off = align_up(off, 256);
    h->off_hj = off; off += h->hj_len * sizeof(double);
    off = align_up(off, 256);
    h->off_grid = off; off += h->grid_len * sizeof(int32_t);
    off = align_up(off, 256);
    h->off_records = off;
    if (r.record_particles) off += (size_t)r.n_particles * sizeof(le_mc_particle);
    // long-first schedule (PLANES and POROUS): list + bitmap of long-lived particles
    const bool long_first = g->desc.kind != LE_MC_GEOM_BULK &&
                            (r.schedule == 1 || (r.schedule == 0 && r.n_particles >= 4096));
    if (long_first && r.n_particles > 0) {
        h->long_cap = (uint32_t)(r.n_particles < (1ull << 20) ? r.n_particles : (1ull << 20));
        h->ext_cap = r.n_particles > kExtMaxParticles ? 0u : (uint32_t)(r.n_particles < kExtCap ? r.n_particles : kExtCap);
        off = align_up(off, 256);
        h->off_long_list = off; off += (size_t)(h->ext_cap + h->long_cap) * sizeof(uint32_t);
        off = align_up(off, 256);
        h->off_long_bits = off; off += (size_t)((r.n_particles + 31) / 32) * sizeof(uint32_t);
        off = align_up(off, 256);
        h->off_long_count = off; off += 4 * sizeof(unsigned int);
    }
    h->dev_bytes = align_up(off, 256);

    cudaError_t e = cudaEventCreate(&h->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_mid);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_stop);
    if (e == cudaSuccess) e = alloc_async((void**)&h->dev, h->dev_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dev, 0, h->dev_bytes, h->stream);
    if (e != cudaSuccess) {
        le_mc_destroy_run(h);
        return cuda_fail(e, "le_mc_run: allocation");
    }
    m->refs.fetch_add(1);
    g->refs.fetch_add(1);
    h->mat = m;
    h->geo = g;

    KernelArgs a;
    memset(&a, 0, sizeof(a));
    TraceParams& P = a.p;
    const bool fp32 = r.precision == LE_MC_PREC_FP32;
    MaterialView mv{};
    material_view(m, &mv);
    fill_material(P, mv, fp32);
    const le_mc_geometry_desc& G = g->desc;
    fill_geometry(P, G);
    fill_run(P, r);
    P.n_bins_x = r.n_bins_x;
    P.n_batch = profile ? r.n_batch : 1;
    P.map_ny = has_map ? r.map_ny : 0;
    P.map_nz = has_map ? r.map_nz : 0;
    P.prof = reinterpret_cast<double*>(h->dev + h->off_prof);
    P.n_hj = r.n_hj;
    P.hj = reinterpret_cast<double*>(h->dev + h->off_hj);
    P.gx = r.grid_nx;
    P.gy = r.grid_ny;
    P.gz = r.grid_nz;
    P.n_samples = r.n_samples;
    P.sample_dt = r.sample_dt;
    P.t_final = (r.source == LE_MC_SRC_PULSE || r.source == LE_MC_SRC_INITIAL) ? r.t_final : 0.0;
    P.grid = reinterpret_cast<int32_t*>(h->dev + h->off_grid);
    P.records = r.record_particles ? reinterpret_cast<le_mc_particle*>(h->dev + h->off_records) : nullptr;
    P.sums = reinterpret_cast<double*>(h->dev + h->off_sums);
    P.counters = reinterpret_cast<unsigned long long*>(h->dev + h->off_counters);
    P.queue = reinterpret_cast<unsigned int*>(h->dev + h->off_queue);
    P.flags = reinterpret_cast<unsigned int*>(h->dev + h->off_flags);
    P.refill_min = r.refill_min > 0 ? r.refill_min : kDefaultRefillMin;
    P.chunk = r.chunk > 0 ? r.chunk : kDefaultChunk;
    fill_round_keys(a);
    if (h->long_cap > 0) {
        P.long_list = reinterpret_cast<uint32_t*>(h->dev + h->off_long_list);
        P.long_bits = reinterpret_cast<uint32_t*>(h->dev + h->off_long_bits);
        P.long_count = reinterpret_cast<unsigned int*>(h->dev + h->off_long_count);
        P.long_cap = h->long_cap;
        P.ext_cap = h->ext_cap;
        P.lam_cut = r.long_mfp_cut > 0.0 ? r.long_mfp_cut : 32.0 * G.L;
    }
    fill_consts(P);

    // slab profiles and steady maps of FP32 kernels: a per-block FP32 copy in
    // shared memory when it is small enough (the H_j split and FP64 profiles
    // are reduced in global memory); for maps only where it costs no
    // resident warps (checked below)
    bool prof_smem = fp32 && profile && h->prof_len <= (size_t)(has_map ? kMapSmemMax : kProfSmemMax);
    int smem_prof = prof_smem ? (int)h->prof_len : 0;
    // launch shape: persistent grid of (SMs x resident blocks).  By default
    // 512 threads per block, or 256 when that keeps more warps resident (a
    // kernel instance whose registers leave room for only one 512-thread
    // block per SM)
    auto shape_for = [&](int t, size_t* sm_bytes, int* resident) {
        cudaError_t err = fp32 ? smem_trace_f32(G.kind, r.source, profile, m->n_modes, t, smem_prof, 0, sm_bytes)
                               : smem_trace_f64(G.kind, r.source, profile, m->n_modes, t, smem_prof, 0, sm_bytes);
        if (err == cudaSuccess)
            err = fp32 ? occupancy_trace_for_f32(P, profile, t, *sm_bytes, resident)
                       : occupancy_trace_for_f64(P, profile, t, *sm_bytes, resident);
        return err;
    };
    int threads = r.threads_per_block > 0 ? r.threads_per_block : kDefaultThreads;
    if (threads > 512) threads = 512;
    size_t smem = 0;
    int per_sm = 0;
    e = shape_for(threads, &smem, &per_sm);
    if (e == cudaSuccess && r.threads_per_block <= 0) {
        size_t smem2 = 0;
        int per_sm2 = 0;
        e = shape_for(256, &smem2, &per_sm2);
        if (e == cudaSuccess && per_sm2 * 256 > per_sm * threads) {
            threads = 256;
            smem = smem2;
            per_sm = per_sm2;
        }
    }
    if (e == cudaSuccess && prof_smem && has_map) {
        // the map copy must not lower the resident warps of this shape
        const int keep = smem_prof;
        smem_prof = 0;
        size_t smem0 = 0;
        int per_sm0 = 0;
        e = shape_for(threads, &smem0, &per_sm0);
        if (e == cudaSuccess && per_sm0 > per_sm) {
            prof_smem = false;
            smem = smem0;
            per_sm = per_sm0;
        } else {
            smem_prof = keep;
        }
    }
    P.prof_smem = prof_smem ? 1 : 0;
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess && r.blocks_per_sm > 0 && r.blocks_per_sm < per_sm) per_sm = r.blocks_per_sm;
    int blocks = sms * per_sm;
    // no more warps than batches of 32 particles (tiny runs)
    const long long max_blocks = ((long long)r.n_particles + 32LL * (threads / 32) - 1) / (32LL * (threads / 32));
    if (blocks > max_blocks) blocks = (int)max_blocks;
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_start, h->stream);
    if (e == cudaSuccess && blocks > 0 && h->long_cap > 0) {
        e = fp32 ? launch_classify_f32(a, sms * 8, h->stream) : launch_classify_f64(a, sms * 8, h->stream);
        h->launches += 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_mid, h->stream);
    if (e == cudaSuccess && blocks > 0) {
        e = fp32 ? launch_trace_f32(a, G.kind, r.source, profile, blocks, threads, smem, h->stream)
                 : launch_trace_f64(a, G.kind, r.source, profile, blocks, threads, smem, h->stream);
        h->launches += 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_stop, h->stream);
    if (e != cudaSuccess) {
        h->failed = true;
        *out = h;  // caller destroys; the handle reports STATE from now on
        return cuda_fail(e, "le_mc_run: launch");
    }
    *out = h;
    return LE_MC_OK;
}

le_mc_status le_mc_wait(le_mc_run_handle h)
{
    if (!h) return fail(LE_MC_ERR_INVALID, "le_mc_wait: null handle");
    if (h->failed) return fail(LE_MC_ERR_STATE, "le_mc_wait: run failed earlier");
    cudaError_t e = cudaEventSynchronize(h->ev_stop);
    if (e != cudaSuccess) {
        h->failed = true;
        return cuda_fail(e, "le_mc_wait");
    }
    return LE_MC_OK;
}

static le_mc_status fetch_header(le_mc_run_handle h)
{
    if (h->have_header) return LE_MC_OK;
    le_mc_status s = le_mc_wait(h);
    if (s != LE_MC_OK) return s;
    unsigned char tmp[2 * sizeof(double) + CNT_N * sizeof(unsigned long long) + 2 * sizeof(unsigned long long)];
    cudaError_t e = cudaMemcpy(tmp, h->dev, sizeof(tmp), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        h->failed = true;
        return cuda_fail(e, "le_mc_read_tallies: copy");
    }
    memcpy(h->sums, tmp + h->off_sums, sizeof(h->sums));
    memcpy(h->counters, tmp + h->off_counters, sizeof(h->counters));
    memcpy(&h->flags, tmp + h->off_flags, sizeof(h->flags));
    if (h->long_cap > 0 && h->launches > 0) {
        unsigned int cnt[3] = {0, 0, 0};
        e = cudaMemcpy(cnt, h->dev + h->off_long_count, sizeof(cnt), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            h->failed = true;
            return cuda_fail(e, "le_mc_read_tallies: copy");
        }
        // the trace kernel's reading of the two lists (all-or-nothing extreme list)
        const bool overflow = cnt[1] > h->ext_cap;
        h->extreme_traced = overflow ? 0u : cnt[1];
        h->long_listed = (cnt[0] < h->long_cap ? cnt[0] : h->long_cap) + (overflow ? h->ext_cap : 0u);
    }
    h->have_header = true;
    return LE_MC_OK;
}

le_mc_status le_mc_read_tallies(le_mc_run_handle h, le_mc_tallies* out)
{
    if (!h || !out) return fail(LE_MC_ERR_INVALID, "le_mc_read_tallies: null argument");
    le_mc_status s = fetch_header(h);
    if (s != LE_MC_OK) return s;
    memset(out, 0, sizeof(*out));
    normalize(&h->geo->desc, &h->desc, h->mat->sums, h->sums, h->counters, out);
    float ms = 0.0f, pre = 0.0f;
    if (h->launches) {
        cudaEventElapsedTime(&ms, h->ev_mid, h->ev_stop);
        cudaEventElapsedTime(&pre, h->ev_start, h->ev_mid);
    }
    out->kernel_ms = ms;
    out->prepass_ms = pre;
    out->kernel_launches = h->launches;
    out->device_flags = h->flags;
    out->long_listed = h->long_listed;
    out->extreme_traced = h->extreme_traced;
    return LE_MC_OK;
}

le_mc_status le_mc_read_array(le_mc_run_handle h, int32_t which, void* dst, size_t capacity, size_t* written)
{
    if (!h) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: null handle");
    const le_mc_run_desc& r = h->desc;
    size_t bytes = 0;
    switch (which) {
    case LE_MC_ARRAY_T: case LE_MC_ARRAY_T_SE: case LE_MC_ARRAY_Q: case LE_MC_ARRAY_Q_SE:
        if (r.n_bins_x <= 0) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run has no profile");
        bytes = (size_t)r.n_bins_x * sizeof(double);
        break;
    case LE_MC_ARRAY_H: case LE_MC_ARRAY_H_SE:
        if (r.n_hj <= 0) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run has no H_j tally");
        bytes = (size_t)r.n_hj * sizeof(double);
        break;
    case LE_MC_ARRAY_GRID:
        if (h->grid_len == 0) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run has no grid");
        bytes = h->grid_len * sizeof(int32_t);
        break;
    case LE_MC_ARRAY_GRID_T:
    case LE_MC_ARRAY_GRID_T_SE:
        if (h->grid_len == 0) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run has no grid");
        bytes = h->grid_len * sizeof(double);
        break;
    case LE_MC_ARRAY_GRID_TX:
    case LE_MC_ARRAY_GRID_TX_SE:
        if (h->grid_len == 0) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run has no grid");
        bytes = (size_t)r.n_samples * r.grid_nx * sizeof(double);
        break;
    case LE_MC_ARRAY_MAP_T: case LE_MC_ARRAY_MAP_T_SE: case LE_MC_ARRAY_MAP_Q: case LE_MC_ARRAY_MAP_Q_SE:
    case LE_MC_ARRAY_MAP_SOLID: case LE_MC_ARRAY_MAP_T_LOCAL:
        if (r.map_ny <= 0 || r.map_nz <= 0) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run has no maps");
        bytes = (size_t)r.map_ny * r.map_nz * sizeof(double);
        break;
    case LE_MC_ARRAY_PARTICLES:
        if (!r.record_particles) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: run kept no records");
        bytes = (size_t)r.n_particles * sizeof(le_mc_particle);
        break;
    default:
        return fail(LE_MC_ERR_INVALID, "le_mc_read_array: unknown array");
    }
    if (written) *written = bytes;
    if (!dst) return LE_MC_OK;
    if (capacity < bytes) return fail(LE_MC_ERR_INVALID, "le_mc_read_array: capacity too small");
    le_mc_status s = fetch_header(h);
    if (s != LE_MC_OK) return s;
    cudaError_t e = cudaSuccess;
    if (which == LE_MC_ARRAY_GRID) {
        e = cudaMemcpy(dst, h->dev + h->off_grid, bytes, cudaMemcpyDeviceToHost);
    } else if (which == LE_MC_ARRAY_GRID_T || which == LE_MC_ARRAY_GRID_TX || which == LE_MC_ARRAY_GRID_T_SE ||
               which == LE_MC_ARRAY_GRID_TX_SE) {
        std::vector<int32_t> counts(h->grid_len);
        e = cudaMemcpy(counts.data(), h->dev + h->off_grid, h->grid_len * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            le_mc_tallies t;
            memset(&t, 0, sizeof(t));
            normalize(&h->geo->desc, &r, h->mat->sums, h->sums, h->counters, &t);
            double* out = static_cast<double*>(dst);
            const bool se = which == LE_MC_ARRAY_GRID_T_SE || which == LE_MC_ARRAY_GRID_TX_SE;
            if (which == LE_MC_ARRAY_GRID_T || which == LE_MC_ARRAY_GRID_T_SE)
                finalize_grid_t(&h->geo->desc, &r, h->mat->sums, t.E_eff, counts.data(), se ? nullptr : out,
                                se ? out : nullptr);
            else
                finalize_grid_tx(&h->geo->desc, &r, h->mat->sums, t.E_eff, counts.data(), se ? nullptr : out,
                                 se ? out : nullptr);
        }
    } else if (which >= LE_MC_ARRAY_MAP_T && which <= LE_MC_ARRAY_MAP_T_LOCAL) {
        const size_t cells = (size_t)r.map_ny * r.map_nz;
        std::vector<double> raw(h->prof_len), out(5 * cells);
        e = cudaMemcpy(raw.data(), h->dev + h->off_prof, raw.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            finalize_map(&h->geo->desc, &r, h->mat->sums, raw.data(), out.data(), out.data() + cells,
                         out.data() + 2 * cells, out.data() + 3 * cells, out.data() + 4 * cells);
            if (which == LE_MC_ARRAY_MAP_T_LOCAL) {
                // add the imposed linear T_eq(z) - T_0 at each cell's centre
                const le_mc_geometry_desc& G = h->geo->desc;
                const double dz = G.pitch / r.map_nz;
                for (int k = 0; k < r.map_nz; ++k)
                    for (int j = 0; j < r.map_ny; ++j)
                        out[(size_t)k * r.map_ny + j] += ((k + 0.5) * dz - 0.5 * G.pitch) * r.dTdz;
                memcpy(dst, out.data(), bytes);
            } else {
                memcpy(dst, out.data() + (size_t)(which - LE_MC_ARRAY_MAP_T) * cells, bytes);
            }
        }
    } else if (which == LE_MC_ARRAY_PARTICLES) {
        e = cudaMemcpy(dst, h->dev + h->off_records, bytes, cudaMemcpyDeviceToHost);
    } else if (which <= LE_MC_ARRAY_Q_SE) {
        std::vector<double> raw(h->prof_len), T(r.n_bins_x), Tse(r.n_bins_x), q(r.n_bins_x), qse(r.n_bins_x);
        e = cudaMemcpy(raw.data(), h->dev + h->off_prof, raw.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            finalize_profile(&h->geo->desc, &r, h->mat->sums, raw.data(), T.data(), Tse.data(), q.data(), qse.data());
            const double* src = which == LE_MC_ARRAY_T ? T.data() : which == LE_MC_ARRAY_T_SE ? Tse.data()
                              : which == LE_MC_ARRAY_Q ? q.data() : qse.data();
            memcpy(dst, src, bytes);
        }
    } else {
        std::vector<double> raw(h->hj_len), H(r.n_hj), Hse(r.n_hj);
        e = cudaMemcpy(raw.data(), h->dev + h->off_hj, raw.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            const double scale = flux_scale(&h->geo->desc, &r, h->mat->sums, nullptr, nullptr, nullptr);
            finalize_hj(&r, scale, raw.data(), H.data(), Hse.data());
            memcpy(dst, which == LE_MC_ARRAY_H ? H.data() : Hse.data(), bytes);
        }
    }
    if (e != cudaSuccess) {
        h->failed = true;
        return cuda_fail(e, "le_mc_read_array: copy");
    }
    return LE_MC_OK;
}

le_mc_status le_mc_destroy_run(le_mc_run_handle h)
{
    if (!h) return LE_MC_OK;
    // the run's kernels read the material tables: let them finish first
    if (h->ev_stop && h->launches && !h->failed) cudaEventSynchronize(h->ev_stop);
    if (h->dev) {
        // stream-ordered free after the run's work
        if (cudaFreeAsync(h->dev, h->stream) != cudaSuccess) cudaFree(h->dev);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_mid) cudaEventDestroy(h->ev_mid);
    if (h->ev_stop) cudaEventDestroy(h->ev_stop);
    material_release(h->mat);
    geometry_release(h->geo);
    delete h;
    return LE_MC_OK;
}

le_mc_status le_mc_philox(const uint32_t* counters, uint32_t key0, uint32_t key1, uint32_t* out, size_t n)
{
    if (!counters || !out) return fail(LE_MC_ERR_INVALID, "le_mc_philox: null pointer");
    if (n == 0) return LE_MC_OK;
    uint4 *d_in = nullptr, *d_out = nullptr;
    CUDA_TRY(cudaMalloc(&d_in, n * sizeof(uint4)), "le_mc_philox: cudaMalloc");
    cudaError_t e = cudaMalloc(&d_out, n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMemcpy(d_in, counters, n * sizeof(uint4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(d_in, key0, key1, d_out, n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d_in);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(e, "le_mc_philox");
    return LE_MC_OK;
}

le_mc_status le_mc_sample_modes(le_mc_material m, int32_t which, const uint32_t* words, int32_t* modes, size_t n)
{
    if (!m || !words || !modes) return fail(LE_MC_ERR_INVALID, "le_mc_sample_modes: null argument");
    if (which != 0 && which != 1) return fail(LE_MC_ERR_INVALID, "le_mc_sample_modes: which must be 0 or 1");
    if (n == 0) return LE_MC_OK;
    uint32_t* d_w = nullptr;
    int32_t* d_m = nullptr;
    CUDA_TRY(cudaMalloc(&d_w, n * sizeof(uint32_t)), "le_mc_sample_modes: cudaMalloc");
    cudaError_t e = cudaMalloc(&d_m, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_w, words, n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_sample_modes(which ? m->d_alias_scat : m->d_alias_emit, m->n_modes, d_w, d_m, n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(modes, d_m, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d_w);
    cudaFree(d_m);
    if (e != cudaSuccess) return cuda_fail(e, "le_mc_sample_modes");
    return LE_MC_OK;
}

le_mc_status le_mc_device_info(int32_t* sm_count, char* name, size_t name_capacity)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "le_mc_device_info");
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev), "le_mc_device_info");
    if (sm_count) *sm_count = prop.multiProcessorCount;
    if (name && name_capacity) {
        strncpy(name, prop.name, name_capacity - 1);
        name[name_capacity - 1] = '\0';
    }
    return LE_MC_OK;
}

}  // extern "C"
