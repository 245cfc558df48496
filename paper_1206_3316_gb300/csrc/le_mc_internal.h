// Internal definitions shared by the host code and the CUDA kernels of the
// le_mc library.  Not part of the public ABI (see include/le_mc.h).
#pragma once

#include <stdint.h>
#include <vector_types.h>

#include "le_mc.h"

namespace lemc {

// Device-side status bits (OR-ed into a status word, never a trap): the
// LE_MC_FLAG_* values of the public header.
enum : uint32_t {
    FLAG_REJECTION_EXHAUSTED = LE_MC_FLAG_REJECTION_EXHAUSTED,
    FLAG_BAD_LAUNCH = LE_MC_FLAG_BAD_LAUNCH,
    FLAG_DEBUG_BOUNDS = LE_MC_FLAG_DEBUG_BOUNDS,
};

// Test hook for failure handling (le_mc_test_fail_allocation): true when the
// library's next device allocation is to report out of memory.
bool alloc_fault_injected();
void set_alloc_fault(int32_t after);

// Global counters produced by a run (u64 each).
enum { CNT_PARTICLES = 0, CNT_SEGMENTS, CNT_SCATTERS, CNT_WALL, CNT_PERIODIC, CNT_TRUNCATED,
       CNT_ABSORBED, CNT_N };

// Fates recorded per particle (same meaning as le_mc_particle::fate).
enum { FATE_ABSORBED = 0, FATE_MAX_SCATTER = 1, FATE_MAX_EVENTS = 2, FATE_T_FINAL = 3, FATE_MAX_COLLISIONS = 4 };

// Random-stream layout: Philox4x32-10 with key = seed and counter
// (event, block, particle id, instance id).  Event 0 is emission (block 0:
// source-specific word, mode, polar cosine, azimuth; blocks 1..64: position
// rejection loop; blocks 65..128: pulse emission time); flight k >= 1 uses
// (k, 0, pid, inst) for (flight length, mode redraw, polar cosine, azimuth).
constexpr uint32_t kMaxTries = 64;
constexpr uint32_t kTimeBlock0 = 65;

// One instance of a batch (same material, geometry kind, source kind and
// caps as the rest of the batch; its own thickness, drive, size and stream).
struct BatchInstance {
    double L, dT_lo, dT_hi, dTdz;
    double lam_cut;        // long-first threshold for this instance
    uint32_t inst_id;      // 4th Philox counter word
    uint32_t n_particles;
    // the same in FP32 for FP32 kernels: L, |dT_lo|, |dT_hi|, the gradient
    // source's direction factor (-1 if dT/dz > 0, else +1), lam_cut
    float L32, wlo32, whi32, dir32, lam_cut32;
    int32_t sign_lo, sign_hi;  // WALLS: sign of dT_lo, dT_hi
};

// Problem constants in one trajectory precision, converted once on the host
// (fill_consts), so that FP32 kernels never convert a double inside the loop:
// on GB300 the FP64 pipe that executes such conversions is narrow, and a
// conversion there stalls the warp for many cycles.
template <typename R>
struct Consts {
    R L, pitch, half, rad, rad2, Dy, Dz;  // geometry
    R spec_lo, spec_hi, spec_pore;        // PARTIAL walls
    R wlo, whi;                           // WALLS: |dT_lo|, |dT_hi|
    R grad_dir;                           // GRADIENT: -1 if dT/dz > 0, else +1
    R init_lo, init_span;                 // INITIAL: heated layer
    R p_sx, p_st, p_tc, p_y0, p_z0;       // PULSE
    R t_final, sample_dt, lam_cut;
    R inv_dt, gsx, gsy, gsz;              // 1 / sample_dt; grid cells per metre along x, y, z
    R g;                                  // scattering mean cosine (0 isotropic)
    R map_dy, map_dz, map_iy, map_iz;     // steady map cell sizes and cells per metre
};

constexpr int kBatchSmemMax = 512;

// Slab profiles and steady maps of FP32 kernels: FP32 shared-memory copy of
// at most kProfSmemMax entries ([4][n_batch][n_bins_x + 1]) or kMapSmemMax
// entries ([2][n_batch][map_nz][map_ny]; used only where it costs no resident
// warps), each warp draining its share of the entries into the FP64 sums
// every kProfDrainEvery loop iterations.
constexpr int kProfSmemMax = 12288;
constexpr int kMapSmemMax = 8192;
constexpr int kProfDrainEvery = 32;

// Extreme particles: emission mean free path above kExtremeFactor times the
// long-first cut (1024 film thicknesses by default), at most kExtCap per
// launch (the rest join the ordinary long-first list).  They only matter in
// launches short enough for one 4096-segment history to be near-critical
// (~1e7 particles of ~50 segments take about as long on a GB300), so
// launches of more than kExtMaxParticles particles keep none: there the
// warps tracing them apart would cost lanes and save nothing.
constexpr double kExtremeFactor = 32.0;
constexpr uint32_t kExtCap = 512;
constexpr unsigned long long kExtMaxParticles = 1ull << 25;

// Default launch shape of le_mc_run: 512 threads per block, refill idle
// lanes once 4 of a warp's 32 are idle, claim queue positions 256 at a time
// (a GB300 sweep of the 1e7-particle film found this fastest; results do not
// depend on the shape).
constexpr int kDefaultThreads = 512;
constexpr int kDefaultRefillMin = 4;
constexpr int kDefaultChunk = 256;  // batches up to this size accumulate per block in shared memory

struct TraceParams {
    // material tables (device pointers)
    const void* props;        // float2 or double2 [n_modes]: (Lambda_b, v_b)
    const uint2* alias_scat;  // [n_modes] (threshold, alias) for C_b / tau_b
    const uint2* alias_emit;  // [n_modes] (threshold, alias) for C_b v_b
    const uint2* alias_init;  // [n_modes] (threshold, alias) for C_b (initial condition)
    int32_t n_modes;
    double scatter_g;         // relaxation-event direction law: 0 isotropic, else Henyey-Greenstein
    // geometry
    int32_t geom, wall_lo, wall_hi, pore_wall;
    int32_t cells_y, cells_z;
    double L, pitch, radius;
    double spec_lo, spec_hi, spec_pore;  // PARTIAL walls: specular probability
    // source
    int32_t src;
    double dT_lo, dT_hi, dTdz;
    double p_sx, p_st, p_tc, p_y0, p_z0;
    double init_dT, init_x_lo, init_x_hi;
    int32_t sign_lo, sign_hi, init_sign;  // WALLS: sign of dT_lo, dT_hi; INITIAL: of init_dT
    int32_t aniso;                        // scatter_g != 0
    int32_t events_fate;                  // fate reported when max_events ends a particle
    Consts<float> c32;                    // filled by fill_consts from the doubles
    Consts<double> c64;
    // run
    uint32_t n_particles, key0, key1, inst, max_scatter, max_events, max_collisions;
    uint32_t scat_cap;  // max_scatter, or 2^32 - 1 when there is no scattering cap
    // slab profile: [4][n_batch][n_bins_x + 1] (T direct, T difference,
    // q direct, q difference), FP64; or, in pored films, the steady maps
    // [2][n_batch][map_nz][map_ny] (sum of s x time, sum of s x z
    // displacement over each map cell)
    int32_t n_bins_x, n_batch;
    int32_t map_ny, map_nz;
    double* prof;
    // FP32 kernels with a slab profile or steady maps small enough keep a
    // per-block FP32 copy in shared memory that their warps drain into prof
    // (0 = every contribution is reduced into prof directly)
    int32_t prof_smem;
    // flux by scattering index: [2][n_hj] (sum s h, sum h^2)
    int32_t n_hj;
    double* hj;
    // transient counting grid [n_samples][gz][gy][gx], int32
    int32_t gx, gy, gz, n_samples;
    double sample_dt, t_final;
    int32_t* grid;
    // per-particle records (le_mc_particle[n_particles]) or null
    le_mc_particle* records;
    // outputs
    double* sums;                  // [2]: sum s L, sum (s L)^2
    unsigned long long* counters;  // [CNT_N]
    unsigned int* queue;           // [1]: next particle id
    unsigned int* flags;           // [1]
    // long-first schedule: ids of particles whose emission mode has a mean
    // free path above lam_cut, served before the natural order (which then
    // skips the ids flagged in long_bits); long_list == nullptr disables it
    // The first ext_cap entries of long_list hold the extreme particles
    // (mean free path above kExtremeFactor lam_cut), each traced by a warp of
    // its own whose idle lanes compute its random words; the ordinary
    // long-first list follows.  long_count[0] counts the long-first list,
    // [1] the extreme list, [2] is the claim counter of the extreme list.
    uint32_t* long_list;           // [ext_cap + long_cap]
    uint32_t* long_bits;           // [ceil(n_particles / 32)]
    unsigned int* long_count;      // [3]
    uint32_t long_cap, ext_cap;
    double lam_cut;
    // batch mode: queue positions 0 .. offsets[n_instances] - 1 run over the
    // concatenated instances; per-instance sums and counters
    const BatchInstance* instances;
    const unsigned long long* offsets;  // [n_instances + 1]
    int32_t n_instances;
    int32_t refill_min;                 // dead lanes a warp tolerates before refilling (>= 1)
    int32_t chunk;                      // queue positions a warp claims at a time (multiple of 32)
    uint32_t first;                     // particle id of queue position 0 (run mode)
    double* inst_sums;                  // [n_instances][2]
    unsigned long long* inst_counters;  // [n_instances][CNT_N]
};

// Host helpers (le_mc_host.cpp).
int build_mode_table(const le_mc_material_desc* d, double* omega, double* v, double* tau, double* C,
                     int capacity, int* n_modes, const char** why);
int build_alias(const double* w, int n, uint32_t* thr, uint32_t* alias, const char** why);
int check_geometry(const le_mc_geometry_desc* g, const char** why);
int check_run(const le_mc_geometry_desc* g, const le_mc_run_desc* r, int n_modes, const char** why);
// Derived constants (signs, both Consts) from the double fields of P; call
// after every double field is set.
void fill_consts(TraceParams& P);
// FP32 fields of a batch instance from its double fields.
void fill_instance32(BatchInstance& b);

struct MaterialSums {
    double C_tot, Cv_sum;
};

// Device tables of a material, for translation units other than the one
// that owns le_mc_material_s.
struct MaterialView {
    const void* props32;
    const void* props64;
    const uint2* alias_scat;
    const uint2* alias_emit;
    const uint2* alias_init;
    int n_modes;
    int device;
    MaterialSums sums;
    double scatter_g;
};
bool material_view(le_mc_material m, MaterialView* out);
void material_retain(le_mc_material m);
// Marks a material whose tables le_mc_run_noalloc work has read (its release
// then waits for the device before freeing them).
void material_mark_noalloc(le_mc_material m);
void material_drop(le_mc_material m);
le_mc_status set_error(le_mc_status s, const char* what, const char* detail);

// Normalisation of the raw device sums into le_mc_tallies (after the
// algorithm: N = energy / E_eff; Eq. 4: E_eff_dot = P / N).
void normalize(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms,
               const double sums[2], const unsigned long long counters[CNT_N], le_mc_tallies* out);

// Batch-mean slab profiles from the raw [4][B][nb+1] arrays.
void finalize_profile(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms,
                      const double* raw, double* T, double* T_se, double* q, double* q_se);
void finalize_hj(const le_mc_run_desc* r, double scale, const double* raw, double* H, double* H_se);
// Transient grids (Eq. 3): per-cell energy temperature, and the average over
// the solid of each x slab, with their standard errors (either output may be
// null); E_eff is the energy of one particle.
void finalize_grid_t(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms, double E_eff,
                     const int32_t* grid, double* T, double* T_se);
void finalize_grid_tx(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms, double E_eff,
                      const int32_t* grid, double* Tx, double* Tx_se);
// Steady maps of a pored film from the raw [2][n_batch][map_nz][map_ny]
// sums: T - T_eq(z) and the local z flux over the solid of each map cell,
// batch-means standard errors, and the solid fraction (any output may be
// null).
void finalize_map(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms, const double* raw,
                  double* T, double* T_se, double* q, double* q_se, double* solid);
// Solid fraction of each of the ny x nz map cells of a unit cell ([nz][ny]).
void map_solid_fractions(double pitch, double radius, int ny, int nz, double* frac);
// Truncation study of the flux split by scattering index (le_mc_truncation_study).
int truncation_study(const double* H, const double* se, int n, double resolved, int first, le_mc_truncation* out,
                     const char** why);
double truncation_tail(const le_mc_truncation* t, int K);
double flux_scale(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms,
                  double* P_out, double* Vref_out, double* Vsolid_out);

}  // namespace lemc
