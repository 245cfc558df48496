// Host-side assembly of the trace kernels' parameters, shared by le_mc_run,
// the batches and le_mc_run_noalloc: the material, geometry, source and run
// fields that every entry point fills alike.  Device pointers (tallies,
// scratch, queues) and whatever an entry point does differently are set by
// the entry point afterwards, then fill_consts derives the rest.
#pragma once

#include "le_mc_internal.h"
#include "trace_kernel.cuh"

namespace lemc {

inline void fill_material(TraceParams& P, const MaterialView& mv, bool fp32)
{
    P.props = fp32 ? mv.props32 : mv.props64;
    P.alias_scat = mv.alias_scat;
    P.alias_emit = mv.alias_emit;
    P.alias_init = mv.alias_init;
    P.n_modes = mv.n_modes;
    P.scatter_g = mv.scatter_g;
}

inline void fill_geometry(TraceParams& P, const le_mc_geometry_desc& G)
{
    P.geom = G.kind;
    P.wall_lo = G.wall_lo;
    P.wall_hi = G.wall_hi;
    P.pore_wall = G.pore_wall;
    P.spec_lo = G.spec_lo;
    P.spec_hi = G.spec_hi;
    P.spec_pore = G.spec_pore;
    P.cells_y = G.kind == LE_MC_GEOM_POROUS ? G.cells_y : 1;
    P.cells_z = G.kind == LE_MC_GEOM_POROUS ? G.cells_z : 1;
    P.L = G.kind == LE_MC_GEOM_BULK ? 1.0 : G.L;
    P.pitch = G.kind == LE_MC_GEOM_POROUS ? G.pitch : 1.0;
    P.radius = G.kind == LE_MC_GEOM_POROUS ? G.radius : 0.0;
}

// Source, random stream and truncation of a run.
inline void fill_run(TraceParams& P, const le_mc_run_desc& r)
{
    P.src = r.source;
    P.dT_lo = r.dT_lo;
    P.dT_hi = r.dT_hi;
    P.dTdz = r.dTdz;
    P.p_sx = r.pulse_sigma_x;
    P.p_st = r.pulse_sigma_t;
    P.p_tc = r.pulse_t_center;
    P.p_y0 = r.pulse_y0;
    P.p_z0 = r.pulse_z0;
    P.init_dT = r.init_dT;
    P.init_x_lo = r.init_x_lo;
    P.init_x_hi = r.init_x_hi;
    P.n_particles = (uint32_t)r.n_particles;
    P.first = r.first_particle;
    P.key0 = (uint32_t)r.seed;
    P.key1 = (uint32_t)(r.seed >> 32);
    P.inst = r.instance_id;
    P.max_scatter = r.max_scatter;
    P.scat_cap = r.max_scatter > 0u ? r.max_scatter : 0xFFFFFFFFu;
    P.max_events = r.max_events;
    P.max_collisions = r.max_collisions;
}

// The ten Philox4x32-10 round keys of the published key schedule (Salmon et
// al., SC'11): k0 + r 0x9E3779B9, k1 + r 0xBB67AE85, r = 0..9.
inline void fill_round_keys(KernelArgs& a)
{
    for (int i = 0; i < 10; ++i) {
        a.rk.k0[i] = a.p.key0 + (uint32_t)i * 0x9E3779B9u;
        a.rk.k1[i] = a.p.key1 + (uint32_t)i * 0xBB67AE85u;
    }
}

}  // namespace lemc
