// Diagnostic kernels exposed through the C ABI: raw Philox4x32-10 blocks and
// alias-table mode draws, used to check the device generator and samplers
// against the oracle bit for bit and against exact probabilities.
#include <cuda_runtime.h>

#include "device_math.cuh"
#include "le_mc_internal.h"

namespace lemc {

namespace {
__global__ void philox_kernel(const uint4* __restrict__ ctr, RoundKeys rk, uint4* __restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(ctr[i], rk);
}

__global__ void sample_modes_kernel(const uint2* __restrict__ table, uint32_t n_modes,
                                    const uint32_t* __restrict__ words, int32_t* __restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)alias_draw(table, n_modes, words[i]);
}

int grid_for(size_t n)
{
    size_t b = (n + 255) / 256;
    if (b > 65535) b = 65535;
    if (b < 1) b = 1;
    return (int)b;
}
}  // namespace

cudaError_t launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, size_t n, cudaStream_t st)
{
    RoundKeys rk;
    for (int i = 0; i < 10; ++i) {
        rk.k0[i] = k0 + (uint32_t)i * 0x9E3779B9u;
        rk.k1[i] = k1 + (uint32_t)i * 0xBB67AE85u;
    }
    philox_kernel<<<grid_for(n), 256, 0, st>>>(ctr, rk, out, n);
    return cudaGetLastError();
}

cudaError_t launch_sample_modes(const uint2* table, int n_modes, const uint32_t* words, int32_t* out, size_t n,
                                cudaStream_t st)
{
    sample_modes_kernel<<<grid_for(n), 256, 0, st>>>(table, (uint32_t)n_modes, words, out, n);
    return cudaGetLastError();
}

}  // namespace lemc
