// Host build of NVIDIA's curand Philox4x32-10 device function (readable
// header, curand_philox4x32_x.h), used only as an independent check of the
// oracle's own Philox4x32-10.  Reads lines "c0 c1 c2 c3 k0 k1" on stdin and
// prints the four output words per line.
#define QUALIFIERS static inline
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>
#include <cstdio>

int main()
{
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        uint4 c = make_uint4(c0, c1, c2, c3);
        uint2 k = make_uint2(k0, k1);
        uint4 r = curand_Philox4x32_10(c, k);
        std::printf("%u %u %u %u\n", r.x, r.y, r.z, r.w);
    }
    return 0;
}
