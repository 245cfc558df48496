// Host-side logic of the le_mc library: FP64 mode tables, Vose alias tables,
// descriptor validation and the normalisation of raw device sums.
// Nothing here touches a GPU, so it is exercised by the CPU test suite.
#include <math.h>
#include <string.h>

#include <atomic>
#include <limits>
#include <vector>

#include "le_mc_internal.h"

namespace lemc {

namespace {
constexpr double kPi = 3.141592653589793;
constexpr double kHbar = 1.054571817e-34;  // J s
constexpr double kBoltzmann = 1.380649e-23;  // J / K
}  // namespace

// Per-mode tables at T_eq.  For the quadratic dispersion each branch is cut
// at k_max = min(2 pi / a, c1 / (2 |c2|)) (positive group velocity) and split
// into n_bins equal frequency bins evaluated at their centres:
//   v = d omega / dk = sqrt(c1^2 + 4 c2 omega),  k = 2 omega / (c1 + v),
//   D = k^2 / (2 pi^2 v) per branch and volume,
//   C = g D hbar omega (d f_BE / dT) d omega,
//   1 / tau = A omega^4 + B omega^2 T exp(-C_exp / T).
int build_mode_table(const le_mc_material_desc* d, double* omega, double* v, double* tau, double* C,
                     int capacity, int* n_modes, const char** why)
{
    if (!d) { *why = "null material descriptor"; return LE_MC_ERR_INVALID; }
    if (!(d->T_eq > 0.0)) { *why = "T_eq must be > 0"; return LE_MC_ERR_INVALID; }
    if (!(d->scatter_g > -1.0 && d->scatter_g < 1.0)) { *why = "scatter_g must be in (-1, 1)"; return LE_MC_ERR_INVALID; }
    int n = 0;
    if (d->kind == LE_MC_MAT_GRAY) {
        if (!(d->gray_v > 0.0) || !(d->gray_tau > 0.0) || !(d->gray_C > 0.0)) {
            *why = "gray v, tau and C must be > 0";
            return LE_MC_ERR_INVALID;
        }
        n = 1;
        if (omega && capacity >= 1) {
            omega[0] = 0.0; v[0] = d->gray_v; tau[0] = d->gray_tau; C[0] = d->gray_C;
        }
    } else if (d->kind == LE_MC_MAT_QUADRATIC) {
        if (d->n_branch < 1 || d->n_branch > LE_MC_MAX_BRANCHES) { *why = "n_branch out of 1..4"; return LE_MC_ERR_INVALID; }
        if (d->n_bins < 1) { *why = "n_bins must be >= 1"; return LE_MC_ERR_INVALID; }
        if ((long long)d->n_bins * d->n_branch > LE_MC_MAX_MODES) { *why = "too many modes"; return LE_MC_ERR_INVALID; }
        if (!(d->a_lattice > 0.0) || d->A < 0.0 || d->B < 0.0 || !(d->A > 0.0 || d->B > 0.0)) {
            *why = "bad lattice constant or scattering law";
            return LE_MC_ERR_INVALID;
        }
        n = d->n_bins * d->n_branch;
        const double T = d->T_eq;
        for (int br = 0; br < d->n_branch; ++br) {
            const double c1 = d->c1[br], c2 = d->c2[br], g = d->degeneracy[br];
            if (!(c1 > 0.0) || !(g > 0.0)) { *why = "branch needs c1 > 0 and degeneracy > 0"; return LE_MC_ERR_INVALID; }
            double kmax = 2.0 * kPi / d->a_lattice;
            if (c2 < 0.0) {
                const double k_vh = c1 / (2.0 * fabs(c2));
                if (k_vh < kmax) kmax = k_vh;
            }
            const double wmax = c1 * kmax + c2 * kmax * kmax;
            const double dw = wmax / d->n_bins;
            if (!omega || capacity < n) continue;
            for (int b = 0; b < d->n_bins; ++b) {
                const int i = br * d->n_bins + b;
                const double w = (b + 0.5) * dw;
                const double vg = sqrt(c1 * c1 + 4.0 * c2 * w);
                const double k = 2.0 * w / (c1 + vg);
                const double dos = k * k / (2.0 * kPi * kPi * vg);
                const double x = kHbar * w / (kBoltzmann * T);
                const double em1 = expm1(x);
                const double dfdT = x * exp(x) / (em1 * em1 * T);
                omega[i] = w;
                v[i] = vg;
                C[i] = g * dos * kHbar * w * dfdT * dw;
                tau[i] = 1.0 / (d->A * w * w * w * w + d->B * w * w * T * exp(-d->C_exp / T));
            }
        }
    } else if (d->kind == LE_MC_MAT_TABULATED) {
        if (d->n_modes < 1 || d->n_modes > LE_MC_MAX_MODES) { *why = "n_modes out of range"; return LE_MC_ERR_INVALID; }
        if (!d->tab_v || !d->tab_tau || !d->tab_C) { *why = "tabulated arrays missing"; return LE_MC_ERR_INVALID; }
        n = d->n_modes;
        for (int i = 0; i < n; ++i) {
            if (!(d->tab_v[i] > 0.0) || !(d->tab_tau[i] > 0.0) || !(d->tab_C[i] >= 0.0)) {
                *why = "tabulated v, tau must be > 0 and C >= 0";
                return LE_MC_ERR_INVALID;
            }
        }
        if (omega && capacity >= n) {
            for (int i = 0; i < n; ++i) { omega[i] = 0.0; v[i] = d->tab_v[i]; tau[i] = d->tab_tau[i]; C[i] = d->tab_C[i]; }
        }
    } else {
        *why = "unknown material kind";
        return LE_MC_ERR_INVALID;
    }
    *n_modes = n;
    return LE_MC_OK;
}

// Vose's alias method (M. D. Vose, IEEE TSE 17(9), 1991), built in FP64 and
// stored as 32-bit integer thresholds: column j keeps itself when the low
// 32 bits of r n are below threshold[j].
int build_alias(const double* w, int n, uint32_t* thr, uint32_t* alias, const char** why)
{
    if (n < 1 || n > LE_MC_MAX_MODES) { *why = "alias table size out of range"; return LE_MC_ERR_INVALID; }
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(w[i] >= 0.0) || !isfinite(w[i])) { *why = "alias weights must be finite and >= 0"; return LE_MC_ERR_INVALID; }
        total += w[i];
    }
    if (!(total > 0.0) || !isfinite(total)) { *why = "alias weights sum to zero"; return LE_MC_ERR_INVALID; }
    std::vector<double> p(n);
    std::vector<int> small, large;
    small.reserve(n);
    large.reserve(n);
    for (int i = 0; i < n; ++i) {
        p[i] = w[i] * (double)n / total;
        if (p[i] < 1.0) small.push_back(i); else large.push_back(i);
    }
    std::vector<double> prob(n, 1.0);
    for (int i = 0; i < n; ++i) alias[i] = (uint32_t)i;
    while (!small.empty() && !large.empty()) {
        const int l = small.back(); small.pop_back();
        const int g = large.back(); large.pop_back();
        prob[l] = p[l];
        alias[l] = (uint32_t)g;
        p[g] = (p[g] + p[l]) - 1.0;
        if (p[g] < 1.0) small.push_back(g); else large.push_back(g);
    }
    // whatever is left holds probability one up to rounding
    for (int i : large) { prob[i] = 1.0; alias[i] = (uint32_t)i; }
    for (int i : small) { prob[i] = 1.0; alias[i] = (uint32_t)i; }
    for (int i = 0; i < n; ++i) {
        if (prob[i] >= 1.0) { thr[i] = 0xFFFFFFFFu; alias[i] = (uint32_t)i; continue; }
        double t = floor(prob[i] * 4294967296.0 + 0.5);
        if (t < 0.0) t = 0.0;
        if (t > 4294967295.0) t = 4294967295.0;
        thr[i] = (uint32_t)t;
    }
    return LE_MC_OK;
}

template <typename R>
static void fill_one(const TraceParams& P, Consts<R>& c)
{
    c.L = (R)P.L;
    c.pitch = (R)P.pitch;
    c.half = (R)(0.5 * P.pitch);
    c.rad = (R)P.radius;
    c.rad2 = (R)(P.radius * P.radius);
    c.Dy = (R)P.pitch * (R)P.cells_y;
    c.Dz = (R)P.pitch * (R)P.cells_z;
    c.spec_lo = (R)P.spec_lo;
    c.spec_hi = (R)P.spec_hi;
    c.spec_pore = (R)P.spec_pore;
    c.wlo = (R)fabs(P.dT_lo);
    c.whi = (R)fabs(P.dT_hi);
    c.grad_dir = P.dTdz > 0.0 ? R(-1) : R(1);
    c.init_lo = (R)P.init_x_lo;
    c.init_span = (R)(P.init_x_hi - P.init_x_lo);
    c.p_sx = (R)P.p_sx;
    c.p_st = (R)P.p_st;
    c.p_tc = (R)P.p_tc;
    c.p_y0 = (R)P.p_y0;
    c.p_z0 = (R)P.p_z0;
    c.t_final = (R)P.t_final;
    c.sample_dt = (R)P.sample_dt;
    c.lam_cut = (R)P.lam_cut;
    c.inv_dt = P.sample_dt > 0.0 ? (R)(1.0 / P.sample_dt) : R(0);
    c.gsx = P.gx > 0 ? (R)(P.gx / P.L) : R(0);
    c.gsy = P.gy > 0 ? (R)(P.gy / (P.pitch * P.cells_y)) : R(0);
    c.gsz = P.gz > 0 ? (R)(P.gz / (P.pitch * P.cells_z)) : R(0);
    c.g = (R)P.scatter_g;
    c.map_dy = P.map_ny > 0 ? (R)(P.pitch / P.map_ny) : R(0);
    c.map_dz = P.map_nz > 0 ? (R)(P.pitch / P.map_nz) : R(0);
    c.map_iy = P.map_ny > 0 ? (R)(P.map_ny / P.pitch) : R(0);
    c.map_iz = P.map_nz > 0 ? (R)(P.map_nz / P.pitch) : R(0);
}

void fill_consts(TraceParams& P)
{
    P.sign_lo = P.dT_lo >= 0.0 ? 1 : -1;
    P.sign_hi = P.dT_hi >= 0.0 ? 1 : -1;
    P.init_sign = P.init_dT >= 0.0 ? 1 : -1;
    P.aniso = P.scatter_g != 0.0 ? 1 : 0;
    // Without periodic faces (PLANES, BULK) every segment ends in a collision
    // (a relaxation or a wall hit), so a collision cap is a segment cap: fold
    // it into max_events and report the collision fate when it is the one
    // that binds (the kernel then needs no per-segment check for it).
    P.events_fate = FATE_MAX_EVENTS;
    if (P.max_collisions > 0u && P.geom != LE_MC_GEOM_POROUS) {
        if (P.max_collisions <= P.max_events) {
            P.max_events = P.max_collisions;
            P.events_fate = FATE_MAX_COLLISIONS;
        }
        P.max_collisions = 0u;
    }
    fill_one<float>(P, P.c32);
    fill_one<double>(P, P.c64);
}

static std::atomic<int32_t> g_alloc_fault{-1};

void set_alloc_fault(int32_t after) { g_alloc_fault.store(after < 0 ? -1 : after); }

bool alloc_fault_injected()
{
    int32_t v = g_alloc_fault.load();
    while (v >= 0) {
        if (g_alloc_fault.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

void fill_instance32(BatchInstance& b)
{
    b.L32 = (float)b.L;
    b.wlo32 = (float)fabs(b.dT_lo);
    b.whi32 = (float)fabs(b.dT_hi);
    b.dir32 = b.dTdz > 0.0 ? -1.0f : 1.0f;
    b.lam_cut32 = (float)b.lam_cut;
    b.sign_lo = b.dT_lo >= 0.0 ? 1 : -1;
    b.sign_hi = b.dT_hi >= 0.0 ? 1 : -1;
}

int check_geometry(const le_mc_geometry_desc* g, const char** why)
{
    if (!g) { *why = "null geometry descriptor"; return LE_MC_ERR_INVALID; }
    auto wall_ok = [](int w) { return w >= LE_MC_WALL_BLACK && w <= LE_MC_WALL_PARTIAL; };
    auto prob_ok = [](double p) { return p >= 0.0 && p <= 1.0; };
    if (g->kind == LE_MC_GEOM_BULK) return LE_MC_OK;
    if (g->kind != LE_MC_GEOM_PLANES && g->kind != LE_MC_GEOM_POROUS) { *why = "unknown geometry kind"; return LE_MC_ERR_INVALID; }
    if (!(g->L > 0.0) || !isfinite(g->L)) { *why = "thickness L must be > 0"; return LE_MC_ERR_INVALID; }
    if (!wall_ok(g->wall_lo) || !wall_ok(g->wall_hi)) { *why = "unknown wall type"; return LE_MC_ERR_INVALID; }
    if (!prob_ok(g->spec_lo) || !prob_ok(g->spec_hi) || !prob_ok(g->spec_pore)) {
        *why = "specularities must be in [0, 1]";
        return LE_MC_ERR_INVALID;
    }
    if (g->kind == LE_MC_GEOM_POROUS) {
        if (!(g->pitch > 0.0) || !(g->radius >= 0.0) || !(2.0 * g->radius < g->pitch)) {
            *why = "porous geometry needs pitch > 0 and 0 <= 2 radius < pitch";
            return LE_MC_ERR_INVALID;
        }
        if (g->pore_wall != LE_MC_WALL_DIFFUSE && g->pore_wall != LE_MC_WALL_SPECULAR &&
            g->pore_wall != LE_MC_WALL_PARTIAL) {
            *why = "pore walls must be diffuse, specular or partially specular";
            return LE_MC_ERR_INVALID;
        }
        if (g->cells_y < 1 || g->cells_z < 1 || g->cells_y > 65535 || g->cells_z > 65535) {
            *why = "cells_y and cells_z must be in 1..65535";
            return LE_MC_ERR_INVALID;
        }
    }
    return LE_MC_OK;
}

int check_run(const le_mc_geometry_desc* g, const le_mc_run_desc* r, int n_modes, const char** why)
{
    if (!r) { *why = "null run descriptor"; return LE_MC_ERR_INVALID; }
    if (r->precision != LE_MC_PREC_FP64 && r->precision != LE_MC_PREC_FP32) { *why = "unknown precision"; return LE_MC_ERR_INVALID; }
    if (r->n_particles + r->first_particle > 0xFFFFFFFFull) {
        *why = "first_particle + n_particles must be < 2^32";
        return LE_MC_ERR_INVALID;
    }
    if (r->max_events < 1) { *why = "max_events must be >= 1"; return LE_MC_ERR_INVALID; }
    if (n_modes < 1 || n_modes > LE_MC_MAX_MODES) { *why = "bad material"; return LE_MC_ERR_INVALID; }
    switch (r->source) {
    case LE_MC_SRC_WALLS:
        if (g->kind != LE_MC_GEOM_PLANES) { *why = "WALLS source needs PLANES geometry"; return LE_MC_ERR_INVALID; }
        if (!isfinite(r->dT_lo) || !isfinite(r->dT_hi) || (r->dT_lo == 0.0 && r->dT_hi == 0.0)) {
            *why = "WALLS source needs a nonzero wall excess";
            return LE_MC_ERR_INVALID;
        }
        break;
    case LE_MC_SRC_GRADIENT:
        if (!(r->dTdz != 0.0) || !isfinite(r->dTdz)) { *why = "GRADIENT source needs dTdz != 0"; return LE_MC_ERR_INVALID; }
        break;
    case LE_MC_SRC_INITIAL:
        if (g->kind != LE_MC_GEOM_POROUS) { *why = "INITIAL source needs POROUS geometry"; return LE_MC_ERR_INVALID; }
        if (!(r->init_dT != 0.0) || !isfinite(r->init_dT)) { *why = "INITIAL needs init_dT != 0"; return LE_MC_ERR_INVALID; }
        if (!(r->init_x_lo >= 0.0) || !(r->init_x_hi <= g->L) || !(r->init_x_hi > r->init_x_lo)) {
            *why = "INITIAL needs 0 <= init_x_lo < init_x_hi <= L";
            return LE_MC_ERR_INVALID;
        }
        if (r->n_particles > 0x7FFFFFFFull) { *why = "INITIAL n_particles must be < 2^31"; return LE_MC_ERR_INVALID; }
        if (!(r->t_final > 0.0)) { *why = "INITIAL needs t_final > 0"; return LE_MC_ERR_INVALID; }
        break;
    case LE_MC_SRC_PULSE:
        if (g->kind != LE_MC_GEOM_POROUS) { *why = "PULSE source needs POROUS geometry"; return LE_MC_ERR_INVALID; }
        if (!(r->pulse_sigma_x > 0.0) || !(r->pulse_sigma_t > 0.0) || !(r->pulse_energy > 0.0)) {
            *why = "PULSE needs sigma_x, sigma_t and energy > 0";
            return LE_MC_ERR_INVALID;
        }
        if (r->n_particles > 0x7FFFFFFFull) { *why = "PULSE n_particles must be < 2^31"; return LE_MC_ERR_INVALID; }
        if (!(r->t_final > 0.0)) { *why = "PULSE needs t_final > 0"; return LE_MC_ERR_INVALID; }
        break;
    default:
        *why = "unknown source";
        return LE_MC_ERR_INVALID;
    }
    if (r->n_bins_x < 0 || r->n_bins_x > LE_MC_MAX_BINS_X) { *why = "n_bins_x out of range"; return LE_MC_ERR_INVALID; }
    if (r->n_bins_x > 0) {
        if (r->source != LE_MC_SRC_WALLS && !(r->source == LE_MC_SRC_GRADIENT && g->kind == LE_MC_GEOM_PLANES)) {
            *why = "profiles need the WALLS source, or the GRADIENT source between planes";
            return LE_MC_ERR_INVALID;
        }
        if (r->n_batch < 1 || r->n_batch > LE_MC_MAX_BATCH) { *why = "n_batch out of 1..64"; return LE_MC_ERR_INVALID; }
    }
    if (r->map_ny < 0 || r->map_nz < 0 || r->map_ny > LE_MC_MAX_MAP || r->map_nz > LE_MC_MAX_MAP ||
        (r->map_ny > 0) != (r->map_nz > 0)) {
        *why = "map_ny, map_nz must both be 0, or both in 1..LE_MC_MAX_MAP";
        return LE_MC_ERR_INVALID;
    }
    if (r->map_ny > 0) {
        if (g->kind != LE_MC_GEOM_POROUS || r->source != LE_MC_SRC_GRADIENT) {
            *why = "steady maps need the POROUS geometry and the GRADIENT source";
            return LE_MC_ERR_INVALID;
        }
        if (r->n_batch < 1 || r->n_batch > LE_MC_MAX_BATCH) { *why = "n_batch out of 1..64"; return LE_MC_ERR_INVALID; }
    }
    if (r->n_hj < 0 || r->n_hj > LE_MC_MAX_HJ) { *why = "n_hj out of range"; return LE_MC_ERR_INVALID; }
    if (r->n_hj > 0 && (r->source == LE_MC_SRC_PULSE || r->source == LE_MC_SRC_INITIAL)) {
        *why = "the flux split by scattering index (n_hj) is a steady estimator";
        return LE_MC_ERR_INVALID;
    }
    if (r->n_samples < 0 || r->n_samples > (1 << 20)) { *why = "n_samples out of 0..2^20"; return LE_MC_ERR_INVALID; }
    if (r->n_samples > 0) {
        if (r->source != LE_MC_SRC_PULSE && r->source != LE_MC_SRC_INITIAL) {
            *why = "grid samples need the PULSE or INITIAL source";
            return LE_MC_ERR_INVALID;
        }
        if (r->grid_nx < 1 || r->grid_ny < 1 || r->grid_nz < 1 || !(r->sample_dt > 0.0)) {
            *why = "grid needs nx, ny, nz >= 1 and sample_dt > 0";
            return LE_MC_ERR_INVALID;
        }
        const double cells = (double)r->n_samples * r->grid_nx * r->grid_ny * r->grid_nz;
        if (cells > 2.0e9) { *why = "grid too large"; return LE_MC_ERR_INVALID; }
    }
    if (r->threads_per_block != 0 && (r->threads_per_block % 32 != 0 || r->threads_per_block < 32 || r->threads_per_block > 512)) {
        *why = "threads_per_block must be a multiple of 32 in 32..512";
        return LE_MC_ERR_INVALID;
    }
    if (r->blocks_per_sm < 0 || r->blocks_per_sm > 32) { *why = "blocks_per_sm out of range"; return LE_MC_ERR_INVALID; }
    if (r->refill_min < 0 || r->refill_min > 32) { *why = "refill_min out of 0..32"; return LE_MC_ERR_INVALID; }
    if (r->chunk < 0 || r->chunk % 32 != 0 || r->chunk > (1 << 20)) {
        *why = "chunk must be a multiple of 32 up to 2^20";
        return LE_MC_ERR_INVALID;
    }
    if (r->schedule < 0 || r->schedule > 2) { *why = "schedule out of 0..2"; return LE_MC_ERR_INVALID; }
    return LE_MC_OK;
}

// Source power P and the reference volume of the flux average.
//  WALLS: each isothermal wall emits (1/4) sum_b C_b v_b |dT| per unit area
//         (angular integral of V_g cos C_{omega,p} over the half space), and
//         the flux is averaged over the slab thickness.
//  GRADIENT: |Eq. 6| integrated over directions gives (1/2) |dT/dz| sum C v
//         per unit solid volume; the flux is averaged over the reference
//         volume (whole cells, pores included).
double flux_scale(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms,
                  double* P_out, double* Vref_out, double* Vsolid_out)
{
    double P = 0.0, Vref = 1.0, Vsolid = 1.0;
    if (r->source == LE_MC_SRC_WALLS) {
        P = 0.25 * ms.Cv_sum * (fabs(r->dT_lo) + fabs(r->dT_hi));
        Vref = g->L;
        Vsolid = g->L;
    } else if (r->source == LE_MC_SRC_GRADIENT) {
        if (g->kind == LE_MC_GEOM_POROUS) {
            const double cells = (double)g->cells_y * g->cells_z;
            Vref = g->pitch * g->pitch * cells * g->L;
            Vsolid = (g->pitch * g->pitch - kPi * g->radius * g->radius) * cells * g->L;
        } else if (g->kind == LE_MC_GEOM_PLANES) {
            Vref = g->L;
            Vsolid = g->L;
        }
        P = 0.5 * fabs(r->dTdz) * ms.Cv_sum * Vsolid;
    }
    if (P_out) *P_out = P;
    if (Vref_out) *Vref_out = Vref;
    if (Vsolid_out) *Vsolid_out = Vsolid;
    return P / Vref;
}

void normalize(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms,
               const double sums[2], const unsigned long long cnt[CNT_N], le_mc_tallies* out)
{
    const double N = r->n_particles > 0 ? (double)r->n_particles : 1.0;
    double P, Vref, Vsolid;
    const double scale = flux_scale(g, r, ms, &P, &Vref, &Vsolid);
    out->P_total = P;
    out->E_eff_dot = P / N;
    out->E_eff = r->source == LE_MC_SRC_PULSE ? r->pulse_energy / N : 0.0;
    if (r->source == LE_MC_SRC_INITIAL) {
        // deviational energy of the initial condition: C_tot |T_i - T_eq| V (solid part of the layer)
        const double pi = 3.141592653589793;
        const double area = (g->pitch * g->pitch - pi * g->radius * g->radius) * g->cells_y * g->cells_z;
        out->E_eff = ms.C_tot * fabs(r->init_dT) * (r->init_x_hi - r->init_x_lo) * area / N;
    }
    out->C_tot = ms.C_tot;
    out->sum_sL = sums[0];
    out->sum_sL2 = sums[1];
    const double mean = sums[0] / N;
    double var = r->n_particles > 1 ? (sums[1] - N * mean * mean) / (N - 1.0) : 0.0;
    if (var < 0.0) var = 0.0;
    const double se = sqrt(var / N);
    out->flux = scale * mean;
    out->flux_se = scale * se;
    out->kappa = out->kappa_se = out->kappa_solid = 0.0;
    out->psi = out->psi_se = 0.0;
    if (r->source == LE_MC_SRC_GRADIENT) {
        out->kappa = -out->flux / r->dTdz;
        out->kappa_se = out->flux_se / fabs(r->dTdz);
        out->kappa_solid = out->kappa * Vref / Vsolid;
    }
    if (r->source == LE_MC_SRC_WALLS && r->dT_lo != r->dT_hi) {
        const double denom = 0.25 * ms.Cv_sum * (r->dT_lo - r->dT_hi);
        out->psi = out->flux / denom;
        out->psi_se = out->flux_se / fabs(denom);
    }
    out->particles = cnt[CNT_PARTICLES];
    out->segments = cnt[CNT_SEGMENTS];
    out->scatters = cnt[CNT_SCATTERS];
    out->wall_hits = cnt[CNT_WALL];
    out->periodic = cnt[CNT_PERIODIC];
    out->truncated = cnt[CNT_TRUNCATED];
    out->absorbed = cnt[CNT_ABSORBED];
}

// The device accumulates, per batch group, direct per-bin sums and a
// difference array for runs of whole bins; bin k of group b holds
// direct[k] + sum_{j <= k} diff[j].  T_k - T_eq = E_eff_dot sum s t_k /
// (C_tot dx) (energy temperature), q_k = E_eff_dot sum s dx_k / dx.
void finalize_profile(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms,
                      const double* raw, double* T, double* T_se, double* q, double* q_se)
{
    const int nb = r->n_bins_x, B = r->n_batch;
    const size_t stride = (size_t)nb + 1;
    const double dx = g->L / nb;
    double P;
    flux_scale(g, r, ms, &P, nullptr, nullptr);
    const unsigned long long N = r->n_particles;
    std::vector<double> tb((size_t)B * nb), qb((size_t)B * nb);
    for (int b = 0; b < B; ++b) {
        const double* Td = raw + (0 * (size_t)B + b) * stride;
        const double* Tr = raw + (1 * (size_t)B + b) * stride;
        const double* qd = raw + (2 * (size_t)B + b) * stride;
        const double* qr = raw + (3 * (size_t)B + b) * stride;
        double accT = 0.0, accq = 0.0;
        for (int k = 0; k < nb; ++k) {
            accT += Tr[k];
            accq += qr[k];
            tb[(size_t)b * nb + k] = Td[k] + accT;
            qb[(size_t)b * nb + k] = qd[k] + accq;
        }
    }
    for (int k = 0; k < nb; ++k) {
        double sT = 0.0, sq = 0.0, sT2 = 0.0, sq2 = 0.0, totT = 0.0, totq = 0.0;
        for (int b = 0; b < B; ++b) {
            // particles in group b: ids b mod B, or (gradient source) the
            // particle pairs (2q, 2q + 1) with q = b mod B
            double ng = 0.0;
            if (r->source == LE_MC_SRC_GRADIENT) {
                for (unsigned long long e = 0; e < 2; ++e) {
                    const unsigned long long Q = N > e ? (N - e + 1) / 2 : 0;
                    ng += (double)(Q / B + ((unsigned long long)b < Q % B ? 1 : 0));
                }
            } else {
                ng = (double)(N / B + ((unsigned long long)b < N % B ? 1 : 0));
            }
            if (ng <= 0.0) ng = 1.0;
            const double Tg = P / ng * tb[(size_t)b * nb + k] / (ms.C_tot * dx);
            const double qg = P / ng * qb[(size_t)b * nb + k] / dx;
            sT += Tg; sT2 += Tg * Tg; sq += qg; sq2 += qg * qg;
            totT += tb[(size_t)b * nb + k];
            totq += qb[(size_t)b * nb + k];
        }
        const double Nd = N > 0 ? (double)N : 1.0;
        if (T) T[k] = P / Nd * totT / (ms.C_tot * dx);
        if (q) q[k] = P / Nd * totq / dx;
        const double vT = B > 1 ? (sT2 - sT * sT / B) / (B - 1.0) : 0.0;
        const double vq = B > 1 ? (sq2 - sq * sq / B) / (B - 1.0) : 0.0;
        if (T_se) T_se[k] = sqrt((vT > 0.0 ? vT : 0.0) / B);
        if (q_se) q_se[k] = sqrt((vq > 0.0 ? vq : 0.0) / B);
    }
}

// Standard error of an Eq. 3 count n of N particles.  At a sample time a
// particle is in at most one cell (and one x slab), and every particle of the
// transient sources carries the same sign, so each particle adds 0 or its
// sign to n: the unbiased estimate of the variance of that per-particle term,
// times N, is N/(N-1) |n| (1 - |n|/N).
static double count_se(double n, double N)
{
    if (N <= 1.0) return 0.0;
    const double a = fabs(n);
    const double v = a * (1.0 - a / N) * (N / (N - 1.0));
    return v > 0.0 ? sqrt(v) : 0.0;
}

void finalize_grid_t(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms, double E_eff,
                     const int32_t* grid, double* T, double* T_se)
{
    const double Dy = g->pitch * g->cells_y, Dz = g->pitch * g->cells_z;
    const double V_cell = (g->L / r->grid_nx) * (Dy / r->grid_ny) * (Dz / r->grid_nz);
    const double f = E_eff / (ms.C_tot * V_cell);
    const double N = (double)r->n_particles;
    const size_t n = (size_t)r->n_samples * r->grid_nz * r->grid_ny * r->grid_nx;
    for (size_t i = 0; i < n; ++i) {
        if (T) T[i] = f * (double)grid[i];
        if (T_se) T_se[i] = f * count_se((double)grid[i], N);
    }
}

void finalize_grid_tx(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms, double E_eff,
                      const int32_t* grid, double* Tx, double* Tx_se)
{
    const double pi = 3.141592653589793;
    const double solid = (g->pitch * g->pitch - pi * g->radius * g->radius) * g->cells_y * g->cells_z;
    const double f = E_eff / (ms.C_tot * solid * (g->L / r->grid_nx));
    const double N = (double)r->n_particles;
    const size_t plane = (size_t)r->grid_nz * r->grid_ny;
    for (int k = 0; k < r->n_samples; ++k)
        for (int ix = 0; ix < r->grid_nx; ++ix) {
            long long c = 0;
            const int32_t* base = grid + (size_t)k * plane * r->grid_nx + ix;
            for (size_t j = 0; j < plane; ++j) c += base[j * r->grid_nx];
            if (Tx) Tx[(size_t)k * r->grid_nx + ix] = f * (double)c;
            if (Tx_se) Tx_se[(size_t)k * r->grid_nx + ix] = f * count_se((double)c, N);
        }
}

// Area of the disk of radius r about the origin below y = a and z = b, from
// the antiderivative of the chord half-length h(y) = sqrt(r^2 - y^2):
// H(y) = (y h(y) + r^2 asin(y / r)) / 2.  Along y the z-extent below b is
// 2h where h <= b, b + h where -h < b < h, and 0 where b <= -h.
static double disk_corner_area(double a, double b, double r)
{
    if (a <= -r || b <= -r) return 0.0;
    if (a > r) a = r;
    auto H = [r](double y) {
        y = y < -r ? -r : (y > r ? r : y);
        const double h = sqrt(fmax(0.0, r * r - y * y));
        return 0.5 * (y * h + r * r * asin(y / r));
    };
    auto piece = [&](double lo, double hi, bool full) {
        lo = fmax(lo, -r);
        hi = fmin(hi, a);
        if (hi <= lo) return 0.0;
        return full ? 2.0 * (H(hi) - H(lo)) : b * (hi - lo) + (H(hi) - H(lo));
    };
    if (b >= r) return piece(-r, r, true);
    const double yb = sqrt(r * r - b * b);
    if (b >= 0.0) return piece(-r, -yb, true) + piece(-yb, yb, false) + piece(yb, r, true);
    return piece(-yb, yb, false);
}

// Solid area of the map cell [ya, yb] x [za, zb] of a unit cell whose pore
// (radius r) is centred at (c, c): the cell minus its overlap with the disk,
// by inclusion-exclusion of four corner areas.
static double cell_solid_area(double c, double r, double ya, double yb, double za, double zb)
{
    const double full = (yb - ya) * (zb - za);
    if (r <= 0.0) return full;
    const double overlap = disk_corner_area(yb - c, zb - c, r) - disk_corner_area(ya - c, zb - c, r) -
                           disk_corner_area(yb - c, za - c, r) + disk_corner_area(ya - c, za - c, r);
    const double a = full - overlap;
    // a cell whose solid is below 1e-12 of its area counts as empty
    return a > 1e-12 * full ? a : 0.0;
}

void map_solid_fractions(double pitch, double radius, int ny, int nz, double* frac)
{
    const double dy = pitch / ny, dz = pitch / nz, c = 0.5 * pitch;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            frac[(size_t)k * ny + j] = cell_solid_area(c, radius, j * dy, (j + 1) * dy, k * dz, (k + 1) * dz) / (dy * dz);
}

void finalize_map(const le_mc_geometry_desc* g, const le_mc_run_desc* r, const MaterialSums& ms, const double* raw,
                  double* T, double* T_se, double* q, double* q_se, double* solid)
{
    const int ny = r->map_ny, nz = r->map_nz, B = r->n_batch;
    const size_t cells = (size_t)ny * nz;
    double P = 0.0;
    flux_scale(g, r, ms, &P, nullptr, nullptr);
    const unsigned long long N = r->n_particles;
    const double Nd = N > 0 ? (double)N : 1.0;
    std::vector<double> frac(cells);
    map_solid_fractions(g->pitch, g->radius, ny, nz, frac.data());
    const double cell_volume = (g->pitch / ny) * (g->pitch / nz) * g->L * g->cells_y * g->cells_z;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (size_t i = 0; i < cells; ++i) {
        const double V = frac[i] * cell_volume;  // solid volume over the map cell
        double sT = 0, sT2 = 0, sq = 0, sq2 = 0, Tt = 0, qt = 0;
        for (int b = 0; b < B; ++b) {
            // group b holds the particle pairs (2q, 2q + 1) with q = b mod B
            double ng = 0.0;
            for (unsigned long long e = 0; e < 2; ++e) {
                const unsigned long long Q = N > e ? (N - e + 1) / 2 : 0;
                ng += (double)(Q / B + ((unsigned long long)b < Q % B ? 1 : 0));
            }
            if (ng <= 0) ng = 1;
            const double rT = raw[(size_t)b * cells + i], rq = raw[((size_t)B + b) * cells + i];
            const double Tb = P / ng * rT / (ms.C_tot * V), qb = P / ng * rq / V;
            sT += Tb; sT2 += Tb * Tb; sq += qb; sq2 += qb * qb;
            Tt += rT;
            qt += rq;
        }
        const double vT = B > 1 ? (sT2 - sT * sT / B) / (B - 1.0) : 0.0;
        const double vq = B > 1 ? (sq2 - sq * sq / B) / (B - 1.0) : 0.0;
        const bool has = frac[i] > 0.0;
        if (T) T[i] = has ? P / Nd * Tt / (ms.C_tot * V) : nan;
        if (T_se) T_se[i] = has ? sqrt(fmax(vT, 0.0) / B) : nan;
        if (q) q[i] = has ? P / Nd * qt / V : nan;
        if (q_se) q_se[i] = has ? sqrt(fmax(vq, 0.0) / B) : nan;
        if (solid) solid[i] = frac[i];
    }
}

void finalize_hj(const le_mc_run_desc* r, double scale, const double* raw, double* H, double* H_se)
{
    const double N = r->n_particles > 0 ? (double)r->n_particles : 1.0;
    for (int j = 0; j < r->n_hj; ++j) {
        const double m = raw[j] / N;
        double v = r->n_particles > 1 ? (raw[r->n_hj + j] - N * m * m) / (N - 1.0) : 0.0;
        if (v < 0.0) v = 0.0;
        if (H) H[j] = scale * m;
        if (H_se) H_se[j] = scale * sqrt(v / N);
    }
}

// ---- choosing the scattering cap from the flux split (<H_j> discussion) ----
// The paper stops collecting contributions once <H_j> (the flux carried
// between the j-th and (j+1)-th relaxation) is of the order of its own
// statistical uncertainty, and notes that the exponential decay of <H_j>
// keeps the error of such a cap under control.  Reading: K_s is the first j
// with |<H_j>| <= its standard error; the decay is fitted as a geometric law
// |<H_j>| = amp ratio^j by weighted least squares on log |<H_j>| (weights
// 1 / var(log |H_j|) = (H_j / se_j)^2) over the contiguous run of indices
// from `first` on that are resolved to `resolved` standard errors; the flux a
// cap K drops is then the geometric tail sum_{j >= K} = sign amp ratio^K /
// (1 - ratio).
int truncation_study(const double* H, const double* se, int n, double resolved, int first, le_mc_truncation* out,
                     const char** why)
{
    if (!H || !se || !out) { *why = "null pointer"; return LE_MC_ERR_INVALID; }
    if (n < 1 || n > LE_MC_MAX_HJ) { *why = "n out of 1..LE_MC_MAX_HJ"; return LE_MC_ERR_INVALID; }
    if (!(resolved > 0.0)) { *why = "resolved must be > 0"; return LE_MC_ERR_INVALID; }
    if (first < 0) { *why = "first must be >= 0"; return LE_MC_ERR_INVALID; }
    for (int j = 0; j < n; ++j)
        if (!isfinite(H[j]) || !(se[j] >= 0.0)) { *why = "H must be finite and H_se >= 0"; return LE_MC_ERR_INVALID; }
    memset(out, 0, sizeof(*out));
    out->k_s = n;
    for (int j = 0; j < n; ++j)
        if (fabs(H[j]) <= se[j]) { out->k_s = j; break; }
    // weighted least squares of y = c0 + c1 j over the resolved run
    double S = 0, Sx = 0, Sy = 0, Sxx = 0, Sxy = 0, Hsum = 0;
    int m = 0;
    for (int j = first; j < n; ++j) {
        if (!(se[j] > 0.0 && fabs(H[j]) > resolved * se[j])) break;
        const double w = (H[j] / se[j]) * (H[j] / se[j]);
        const double y = log(fabs(H[j]));
        S += w;
        Sx += w * j;
        Sy += w * y;
        Sxx += w * (double)j * j;
        Sxy += w * j * y;
        Hsum += H[j];
        ++m;
    }
    out->n_fit = m;
    out->ratio = std::numeric_limits<double>::quiet_NaN();
    if (m >= 2) {
        const double det = S * Sxx - Sx * Sx;
        if (det > 0.0) {
            const double c1 = (S * Sxy - Sx * Sy) / det;
            const double c0 = (Sy - c1 * Sx) / S;
            out->ratio = exp(c1);
            out->amp = exp(c0);
            out->sign = Hsum > 0.0 ? 1.0 : (Hsum < 0.0 ? -1.0 : 0.0);
        }
    }
    return LE_MC_OK;
}

double truncation_tail(const le_mc_truncation* t, int K)
{
    if (!(t->ratio > 0.0 && t->ratio < 1.0)) return 0.0;
    return t->sign * t->amp * pow(t->ratio, (double)K) / (1.0 - t->ratio);
}

}  // namespace lemc
