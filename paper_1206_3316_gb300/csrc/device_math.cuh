// Device helpers of the trace kernels: the Philox4x32-10 counter-based
// generator and per-precision maths (uniforms, -ln u, sqrt, sincos(2 pi u)).
#pragma once

#include <stdint.h>

namespace lemc {

// Philox4x32-10 from its published definition (Salmon, Moraes, Dror, Shaw,
// SC'11): ten rounds; each multiplies word 0 by 0xD2511F53 and word 2 by
// 0xCD9E8D57 (32x32 -> 64 bits) and mixes the high halves with the other
// words and the round key.  The ten round keys (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85) are precomputed on the host and passed as kernel
// parameters, so they are read from the constant bank by the XORs.
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys& rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
    }
    return c;
}

// The random words of one flight of one particle: Philox4x32-10 of counter
// (n, 0, pid, inst).  The first round's product of the pid word and the
// words it meets there (the zero word, the instance word, the first round
// keys) do not change along a history, so they are formed once per particle
// (philox_lane) and each flight starts from them (philox_flight): one
// multiplication and one XOR fewer per flight, the same words.
struct PhiloxLane {
    uint32_t a;  // mulhi(0xCD9E8D57, pid) ^ 0 ^ k0[0]
    uint32_t b;  // mullo(0xCD9E8D57, pid)
    uint32_t c;  // inst ^ k1[0]
};

__device__ __forceinline__ PhiloxLane philox_lane(uint32_t pid, uint32_t inst, const RoundKeys& rk)
{
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * pid;
    PhiloxLane l;
    l.a = (uint32_t)(p1 >> 32) ^ rk.k0[0];
    l.b = (uint32_t)p1;
    l.c = inst ^ rk.k1[0];
    return l;
}

__device__ __forceinline__ uint4 philox_flight(uint32_t n, const PhiloxLane& l, const RoundKeys& rk)
{
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * n;
    uint4 c = make_uint4(l.a, l.b, (uint32_t)(p0 >> 32) ^ l.c, (uint32_t)p0);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const unsigned long long q0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long q1 = (unsigned long long)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(q0 >> 32), lo0 = (uint32_t)q0;
        const uint32_t hi1 = (uint32_t)(q1 >> 32), lo1 = (uint32_t)q1;
        c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
    }
    return c;
}

template <typename R>
struct DMath;

// FP32 trajectories.  Uniform u = ((r >> 9) + 1/2) 2^-23 in ]0,1[ (built
// from the bit pattern 1.m - (1 - 2^-24), exact); -ln u through the MUFU
// base-2 logarithm; sincos of 2 pi u evaluated on [-pi, pi[ and reflected.
template <>
struct DMath<float> {
    static __device__ __forceinline__ float uniform(uint32_t r)
    {
        return __int_as_float(0x3F800000u | (r >> 9)) - 0.99999994f;
    }
    static __device__ __forceinline__ float neg_log(float u) { return -0.693147180559945f * __log2f(u); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
    static __device__ __forceinline__ void sincos_2pi(float u, float* s, float* c)
    {
        float sn, cs;
        __sincosf(fmaf(u, 6.28318530717958648f, -3.14159265358979324f), &sn, &cs);
        *s = -sn;
        *c = -cs;
    }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
    static __device__ __forceinline__ float big() { return 3.0e38f; }
    // The value of x as a double, assembled from its bits on the integer
    // units: GB300's FP64 units are narrow (a conversion there costs a warp
    // as much as dozens of FP32 operations), and an FP32 kernel only needs
    // the exact widening for its FP64 tally reductions.  Exact for zeros,
    // normal numbers, infinities and NaNs; a subnormal (which these kernels
    // flush to zero, -ftz=true) would be mis-scaled.
    static __device__ __forceinline__ double to_f64(float x)
    {
        const uint32_t u = __float_as_uint(x);
        const uint32_t sgn = u & 0x80000000u, mag = u & 0x7FFFFFFFu;
        // exponent rebias 127 -> 1023 is + 896 in the exponent field
        uint32_t hi = sgn | ((mag >> 3) + (896u << 20));
        hi = mag == 0u ? sgn : hi;
        hi = mag >= 0x7F800000u ? (sgn | 0x7FF00000u | ((mag >> 3) & 0x000FFFFFu)) : hi;
        const uint32_t lo = mag == 0u ? 0u : (u << 29);
        return __hiloint2double((int)hi, (int)lo);
    }
};

// FP64 trajectories: u = (r + 1/2) 2^-32 and the CUDA maths library.
template <>
struct DMath<double> {
    static __device__ __forceinline__ double uniform(uint32_t r)
    {
        // r 2^-32 + 2^-33 in one fused multiply-add: every step is exact,
        // so the value is (r + 1/2) 2^-32 to the bit
        return fma((double)r, 1.0 / 4294967296.0, 1.0 / 8589934592.0);
    }
    static __device__ __forceinline__ double neg_log(double u) { return -log(u); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
    // sin and cos of 2 pi u as sincospi(2u): the argument needs no range
    // reduction (measured 5.7 % faster on the FP64 gray slab than cos and
    // sin of the product 2 pi u; the two agree to the last bit or so)
    static __device__ __forceinline__ void sincos_2pi(double u, double* s, double* c)
    {
        sincospi(2.0 * u, s, c);
    }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
    static __device__ __forceinline__ double big() { return 1.0e300; }
    static __device__ __forceinline__ double to_f64(double x) { return x; }
};

// Mode draw from an alias table: column j = floor(r n / 2^32), kept when the
// low word of r n is below its threshold, else its alias.
__device__ __forceinline__ uint32_t alias_draw(const uint2* table, uint32_t n, uint32_t r)
{
    const unsigned long long m = (unsigned long long)r * n;
    const uint32_t j = (uint32_t)(m >> 32);
    const uint2 e = table[j];
    return ((uint32_t)m < e.x) ? j : e.y;
}

}  // namespace lemc
