// Device-side layout shared by the request server (le_mc_server.cu) and its
// resident trace kernel (serve_kernel.cu).  Internal; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device_math.cuh"
#include "le_mc_internal.h"

namespace lemc {

// Families the resident kernel traces: (geometry, source) pairs with FP32
// trajectories, isotropic relaxation events and black / diffuse / specular
// walls (diffuse or specular pores).
enum { SERVE_SLAB = 0,    // PLANES, WALLS source (slab between isothermal walls)
       SERVE_FILM = 1,    // PLANES, GRADIENT source (film, in-plane conductivity)
       SERVE_POROUS = 2,  // POROUS, GRADIENT source (pored film)
       SERVE_BULK = 3 };  // BULK, GRADIENT source

// One admitted request, in device memory from admission to retirement.
struct ServeSlot {
    TraceParams p;        // the run's parameters (material tables, geometry, source, caps, stream)
    RoundKeys rk;         // Philox4x32-10 round keys of its seed
    const uint4* fused;   // its Eq. 2 table: (threshold, alias, Lambda_j ln 2, Lambda_alias ln 2) in FP32 bits
    int32_t family;       // SERVE_*
    int32_t pad;
};

// A request's running totals (zeroed at admission): the Eq. 4 sums, the
// counters, the status bits, and how many particles they include.
struct ServeTally {
    double sums[2];
    unsigned long long counters[CNT_N];
    unsigned long long done;
    unsigned int flags;
    unsigned int pad;
};

// A work item: particle ids first .. first + count - 1 of the request in slot.
struct ServeItem {
    uint32_t slot, first, count, pad;
};

// Host-written control block, in mapped pinned host memory: the number of
// items published (items are written before it is advanced) and the stop word.
struct ServeControl {
    unsigned long long tail;
    unsigned int stop;
    unsigned int pad;
};

struct ServeArgs {
    ServeSlot* slots;               // device [n_slots]
    ServeTally* tallies;            // device [n_slots]
    const ServeItem* items;         // mapped host ring [ring_mask + 1]
    const unsigned long long* tail; // mapped host: items published
    const unsigned int* stop;       // mapped host: leave the kernel when nonzero
    unsigned long long* head;       // device: items claimed
    unsigned int* status;           // device: LE_MC_FLAG_BAD_LAUNCH if the kernel met a bad launch or item
    uint32_t ring_mask;             // ring capacity - 1 (a power of two)
    uint32_t n_slots;
    unsigned long long idle_ns;     // a warp leaves after finding no work for this long
};

cudaError_t serve_occupancy(int threads, int* per_sm);
cudaError_t launch_serve(const ServeArgs& a, int blocks, int threads, cudaStream_t st);

}  // namespace lemc
