// le_mc_run_noalloc: the trace kernel for callers that must not allocate
// GPU memory.
//
// Who needs it: code that runs where device allocation is unavailable or
// forbidden, e.g. inside a host callback or a region that a framework's own
// memory manager owns (cudaMalloc / cudaMallocAsync calls there would fail,
// deadlock or break the manager's accounting), or a latency-critical loop
// that cannot afford an allocator call.  Such a caller prepares the material
// and geometry beforehand and passes its own device buffers for the results;
// this entry point then calls no cudaMalloc, cudaMallocAsync, cudaFree or
// allocating library routine, and creates no event or stream.
//
// The kernel's scratch memory (particle queue head, warning flags and the
// long-first list and bitmap) lives in one file-scope device array,
// g_noalloc_scratch, of fixed size.  Every GPU that loads the library holds
// it until the process exits.  Its device address is looked up once per
// device with cudaGetSymbolAddress (host code never uses the symbol itself
// as a device pointer); that lookup happens inside the first call on each
// device, so that first call should be made before any stream capture.
// All calls share the array: calls whose device work overlaps in time (on
// different streams, or from different host threads) race on it and must
// be serialised by the caller.  The cached address belongs to the device
// context that existed at the first call; after cudaDeviceReset it is stale,
// so the library must not be used across a reset.
//
// The kernels hold no reference on the material (taking one would allocate
// nothing, but releasing it would need a completion callback or event that
// this entry point may not create), so the material is marked instead and
// le_mc_destroy_material waits for the whole device before freeing its
// tables.  Device status bits of the last call stay in the array and are
// read back with le_mc_noalloc_flags.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "le_mc_internal.h"
#include "trace_kernel.cuh"
#include "le_mc_params.h"

namespace lemc {
cudaError_t launch_trace_f32(const KernelArgs& a, int geom, int src, bool profile, int blocks, int threads,
                             size_t smem, cudaStream_t st);
cudaError_t launch_trace_f64(const KernelArgs& a, int geom, int src, bool profile, int blocks, int threads,
                             size_t smem, cudaStream_t st);
cudaError_t occupancy_trace_for_f32(const TraceParams& p, bool profile, int threads, size_t smem, int* per_sm);
cudaError_t occupancy_trace_for_f64(const TraceParams& p, bool profile, int threads, size_t smem, int* per_sm);
cudaError_t smem_trace_f32(int geom, int src, bool profile, int n_modes, int threads, int prof_len, int hj_len,
                           size_t* bytes);
cudaError_t smem_trace_f64(int geom, int src, bool profile, int n_modes, int threads, int prof_len, int hj_len,
                           size_t* bytes);
cudaError_t launch_classify_f32(const KernelArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_classify_f64(const KernelArgs& a, int blocks, cudaStream_t st);
le_mc_status set_cuda_error(cudaError_t e, const char* where);
bool geometry_view(le_mc_geometry g, le_mc_geometry_desc* out);
}  // namespace lemc

using namespace lemc;

namespace {

// Scratch layout (bytes): [0, 8) queue head, [8, 12) flags, [16, 28) the
// long-first and extreme-list counts and the extreme-list claim counter, then
// the extreme and long-first lists and the bitmap of listed particles.
constexpr size_t kHeader = 256;
constexpr uint32_t kListCap = 1u << 14;
constexpr uint32_t kNoallocExtCap = kExtCap;
constexpr size_t kListBytes = (size_t)(kNoallocExtCap + kListCap) * sizeof(uint32_t);
constexpr size_t kBitsBytes = (size_t)(LE_MC_NOALLOC_MAX_PARTICLES / 32) * sizeof(uint32_t);
constexpr size_t kScratchBytes = kHeader + kListBytes + kBitsBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

le_mc_status le_mc_run_noalloc(le_mc_material m, le_mc_geometry g, const le_mc_run_desc* desc, double* d_sums,
                               unsigned long long* d_counters, void* stream)
{
    if (!m || !g || !desc || !d_sums || !d_counters)
        return set_error(LE_MC_ERR_INVALID, "le_mc_run_noalloc", "null argument");
    MaterialView mv{};
    le_mc_geometry_desc G;
    if (!material_view(m, &mv) || !geometry_view(g, &G))
        return set_error(LE_MC_ERR_INVALID, "le_mc_run_noalloc", "bad handle");
    const char* why = "";
    if (check_run(&G, desc, mv.n_modes, &why) != LE_MC_OK) return set_error(LE_MC_ERR_INVALID, "le_mc_run_noalloc", why);
    const le_mc_run_desc& r = *desc;
    if (r.n_particles > LE_MC_NOALLOC_MAX_PARTICLES)
        return set_error(LE_MC_ERR_INVALID, "le_mc_run_noalloc",
                         "n_particles above LE_MC_NOALLOC_MAX_PARTICLES (trace larger problems in pieces with "
                         "first_particle)");
    if (r.source == LE_MC_SRC_PULSE || r.source == LE_MC_SRC_INITIAL || r.n_bins_x > 0 || r.n_hj > 0 || r.record_particles ||
        r.map_ny > 0)
        return set_error(LE_MC_ERR_INVALID, "le_mc_run_noalloc",
                         "only the scalar sums and counters are produced (no grid, profile, H_j or records)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_run_noalloc");
    if (dev != mv.device) return set_error(LE_MC_ERR_INVALID, "le_mc_run_noalloc", "material lives on another device");
    unsigned char* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_run_noalloc: cudaGetSymbolAddress");
    cudaStream_t st = (cudaStream_t)stream;
    material_mark_noalloc(m);
    const bool fp32 = r.precision == LE_MC_PREC_FP32;
    const uint64_t N = r.n_particles;
    const bool long_first = G.kind != LE_MC_GEOM_BULK && r.schedule != 2 && N >= 4096;

    // results start at zero; so do the queue head, flags, count and the bitmap words in use
    e = cudaMemsetAsync(d_sums, 0, 2 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counters, 0, CNT_N * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, 32, st);
    if (e == cudaSuccess && long_first) e = cudaMemsetAsync(scratch + kHeader + kListBytes, 0, (size_t)((N + 31) / 32) * 4, st);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_run_noalloc: clear");

    KernelArgs a;
    memset(&a, 0, sizeof(a));
    TraceParams& P = a.p;
    fill_material(P, mv, fp32);
    fill_geometry(P, G);
    fill_run(P, r);
    P.n_particles = (uint32_t)N;
    P.n_batch = 1;
    P.sums = d_sums;
    P.counters = d_counters;
    P.queue = reinterpret_cast<unsigned int*>(scratch);
    P.flags = reinterpret_cast<unsigned int*>(scratch + 8);
    if (long_first) {
        P.long_count = reinterpret_cast<unsigned int*>(scratch + 16);
        P.long_list = reinterpret_cast<uint32_t*>(scratch + kHeader);
        P.long_bits = reinterpret_cast<uint32_t*>(scratch + kHeader + kListBytes);
        P.long_cap = kListCap;
        P.ext_cap = kNoallocExtCap;
        P.lam_cut = r.long_mfp_cut > 0.0 ? r.long_mfp_cut : 32.0 * G.L;
    }
    P.refill_min = r.refill_min > 0 ? r.refill_min : 1;
    P.chunk = r.chunk > 0 ? r.chunk : 32;
    fill_consts(P);
    fill_round_keys(a);

    int threads = r.threads_per_block > 0 ? r.threads_per_block : 256;
    size_t smem = 0;
    e = fp32 ? smem_trace_f32(G.kind, r.source, false, mv.n_modes, threads, 0, 0, &smem)
             : smem_trace_f64(G.kind, r.source, false, mv.n_modes, threads, 0, 0, &smem);
    int sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = fp32 ? occupancy_trace_for_f32(P, false, threads, smem, &per_sm)
                 : occupancy_trace_for_f64(P, false, threads, smem, &per_sm);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess && r.blocks_per_sm > 0 && r.blocks_per_sm < per_sm) per_sm = r.blocks_per_sm;
    int blocks = sms * per_sm;
    const long long max_blocks = ((long long)N + 32LL * (threads / 32) - 1) / (32LL * (threads / 32));
    if (blocks > max_blocks) blocks = (int)max_blocks;
    if (e == cudaSuccess && blocks > 0 && long_first)
        e = fp32 ? launch_classify_f32(a, sms * 8, st) : launch_classify_f64(a, sms * 8, st);
    if (e == cudaSuccess && blocks > 0)
        e = fp32 ? launch_trace_f32(a, G.kind, r.source, false, blocks, threads, smem, st)
                 : launch_trace_f64(a, G.kind, r.source, false, blocks, threads, smem, st);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_run_noalloc: launch");
    return LE_MC_OK;
}

le_mc_status le_mc_noalloc_flags(void* stream, uint32_t* flags)
{
    if (!flags) return set_error(LE_MC_ERR_INVALID, "le_mc_noalloc_flags", "null argument");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_noalloc_flags");
    unsigned char* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_noalloc_flags: cudaGetSymbolAddress");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t word = 0;
    // a pageable destination: the copy is complete when cudaMemcpyAsync
    // returns; the stream synchronisation makes that explicit
    e = cudaMemcpyAsync(&word, scratch + 8, sizeof(word), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(e, "le_mc_noalloc_flags: copy");
    *flags = word;
    return LE_MC_OK;
}

}  // extern "C"
