// Instantiations and launchers of the trace kernels in one trajectory
// precision.  The build compiles this file twice, with LEMC_PREC_BITS=32
// (float kernels, launchers named *_f32) and LEMC_PREC_BITS=64 (double
// kernels, *_f64), so the two precisions compile in parallel from one source.
#include <cuda_runtime.h>

#include "trace_kernel.cuh"

#if !defined(LEMC_PREC_BITS)
#error "compile with -DLEMC_PREC_BITS=32 or -DLEMC_PREC_BITS=64"
#elif LEMC_PREC_BITS == 32
using Real = float;
#define LEMC_NAME(fn) fn##_f32
#elif LEMC_PREC_BITS == 64
using Real = double;
#define LEMC_NAME(fn) fn##_f64
#else
#error "LEMC_PREC_BITS must be 32 or 64"
#endif

namespace lemc {

namespace {
template <int G, int S, bool PR, bool DF = false>
cudaError_t launch_one(const KernelArgs& a, int blocks, int threads, size_t smem, cudaStream_t st)
{
    auto k = trace_entry<Real, G, S, PR, false, DF>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks <= 0) return cudaSuccess;
    k<<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int G, int S, bool PR, bool DF = false>
cudaError_t occupancy_one(int threads, size_t smem, int* per_sm)
{
    auto k = trace_entry<Real, G, S, PR, false, DF>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
}

template <int G, int S, bool PR>
cudaError_t smem_one(int n_modes, int threads, int prof_len, int hj_len, size_t* bytes)
{
    *bytes = trace_smem_bytes<Real, G, S, PR>(n_modes, threads, prof_len, hj_len);
    return cudaSuccess;
}
}  // namespace

// Valid (geometry, source, profile) combinations; anything else is rejected
// by the host validation before a launch is attempted.
#define LEMC_DISPATCH(FN, ...)                                                                      \
    if (geom == LE_MC_GEOM_PLANES && src == LE_MC_SRC_WALLS && profile)                              \
        return FN<LE_MC_GEOM_PLANES, LE_MC_SRC_WALLS, true>(__VA_ARGS__);                            \
    if (geom == LE_MC_GEOM_PLANES && src == LE_MC_SRC_WALLS)                                         \
        return FN<LE_MC_GEOM_PLANES, LE_MC_SRC_WALLS, false>(__VA_ARGS__);                           \
    if (geom == LE_MC_GEOM_PLANES && src == LE_MC_SRC_GRADIENT && profile)                           \
        return FN<LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, true>(__VA_ARGS__);                         \
    if (geom == LE_MC_GEOM_PLANES && src == LE_MC_SRC_GRADIENT)                                      \
        return FN<LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false>(__VA_ARGS__);                        \
    if (geom == LE_MC_GEOM_BULK && src == LE_MC_SRC_GRADIENT)                                        \
        return FN<LE_MC_GEOM_BULK, LE_MC_SRC_GRADIENT, false>(__VA_ARGS__);                          \
    if (geom == LE_MC_GEOM_POROUS && src == LE_MC_SRC_GRADIENT && profile)                           \
        return FN<LE_MC_GEOM_POROUS, LE_MC_SRC_GRADIENT, true>(__VA_ARGS__);                         \
    if (geom == LE_MC_GEOM_POROUS && src == LE_MC_SRC_GRADIENT)                                      \
        return FN<LE_MC_GEOM_POROUS, LE_MC_SRC_GRADIENT, false>(__VA_ARGS__);                        \
    if (geom == LE_MC_GEOM_POROUS && src == LE_MC_SRC_PULSE)                                         \
        return FN<LE_MC_GEOM_POROUS, LE_MC_SRC_PULSE, false>(__VA_ARGS__);                           \
    if (geom == LE_MC_GEOM_POROUS && src == LE_MC_SRC_INITIAL)                                       \
        return FN<LE_MC_GEOM_POROUS, LE_MC_SRC_INITIAL, false>(__VA_ARGS__);                         \
    return cudaErrorInvalidValue;

// Films and porous films driven by a gradient with every wall diffuse use
// the DIFF specialisation (same arithmetic, no wall-type lookups).
static bool all_diffuse(const TraceParams& p)
{
    return p.src == LE_MC_SRC_GRADIENT && (p.geom == LE_MC_GEOM_PLANES || p.geom == LE_MC_GEOM_POROUS) &&
           p.wall_lo == LE_MC_WALL_DIFFUSE && p.wall_hi == LE_MC_WALL_DIFFUSE &&
           (p.geom != LE_MC_GEOM_POROUS || p.pore_wall == LE_MC_WALL_DIFFUSE) && p.aniso == 0 && p.n_hj == 0;
}

cudaError_t LEMC_NAME(launch_trace)(const KernelArgs& a, int geom, int src, bool profile, int blocks, int threads,
                              size_t smem, cudaStream_t st)
{
    if (all_diffuse(a.p) && !profile) {
        if (geom == LE_MC_GEOM_PLANES)
            return launch_one<LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true>(a, blocks, threads, smem, st);
        return launch_one<LE_MC_GEOM_POROUS, LE_MC_SRC_GRADIENT, false, true>(a, blocks, threads, smem, st);
    }
    LEMC_DISPATCH(launch_one, a, blocks, threads, smem, st)
}

cudaError_t LEMC_NAME(occupancy_trace)(int geom, int src, bool profile, int threads, size_t smem, int* per_sm)
{
    LEMC_DISPATCH(occupancy_one, threads, smem, per_sm)
}

// Occupancy of the kernel that launch_trace picks for these parameters.
cudaError_t LEMC_NAME(occupancy_trace_for)(const TraceParams& p, bool profile, int threads, size_t smem, int* per_sm)
{
    if (all_diffuse(p) && !profile) {
        if (p.geom == LE_MC_GEOM_PLANES)
            return occupancy_one<LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true>(threads, smem, per_sm);
        return occupancy_one<LE_MC_GEOM_POROUS, LE_MC_SRC_GRADIENT, false, true>(threads, smem, per_sm);
    }
    return LEMC_NAME(occupancy_trace)(p.geom, p.src, profile, threads, smem, per_sm);
}

cudaError_t LEMC_NAME(smem_trace)(int geom, int src, bool profile, int n_modes, int threads, int prof_len, int hj_len,
                            size_t* bytes)
{
    LEMC_DISPATCH(smem_one, n_modes, threads, prof_len, hj_len, bytes)
}

// Batch mode: PLANES geometry with the WALLS or GRADIENT source.
cudaError_t LEMC_NAME(batch_attr)(int src, bool diff, int threads, size_t smem, int* per_sm)
{
    auto k = src == LE_MC_SRC_WALLS ? trace_entry<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_WALLS, false, true>()
             : diff                 ? trace_entry<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true, true>()
                                    : trace_entry<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
}

// Launch only (no attribute calls), so it can be captured into a graph.
cudaError_t LEMC_NAME(batch_launch)(const KernelArgs& a, int src, bool diff, int blocks, int threads, size_t smem,
                              cudaStream_t st)
{
    if (blocks <= 0) return cudaSuccess;
    if (src == LE_MC_SRC_WALLS)
        trace_entry<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_WALLS, false, true>()<<<blocks, threads, smem, st>>>(a);
    else if (diff)
        trace_entry<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true, true>()<<<blocks, threads, smem, st>>>(a);
    else
        trace_entry<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true>()<<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

size_t LEMC_NAME(batch_smem)(int src, int n_modes, int threads, int n_instances)
{
    return src == LE_MC_SRC_WALLS
               ? trace_smem_bytes<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_WALLS, false, true>(n_modes, threads, 0, 0, n_instances)
               : trace_smem_bytes<Real, LE_MC_GEOM_PLANES, LE_MC_SRC_GRADIENT, false, true>(n_modes, threads, 0, 0,
                                                                                            n_instances);
}

cudaError_t LEMC_NAME(launch_classify)(const KernelArgs& a, int blocks, cudaStream_t st)
{
    classify_kernel<Real><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace lemc
