/*
 * le_mc_oracle.c -- plain, slow, FP64 CPU oracle for the linearized
 * energy-based deviational Monte Carlo method of Peraud & Hadjiconstantinou,
 * "An alternative approach to efficient simulation of micro/nanoscale phonon
 * transport" (arXiv:1206.3316).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  The product (the CUDA
 * library under paper_1206_3316_gb300/) shares no code with it.
 *
 * Every particle is traced alone, one step of the paper's trajectory algorithm
 * (steps I-VI) at a time, in FP64, with no blocking, batching or reordering.
 * Mode draws use a plain inverse-CDF search (not alias tables).
 *
 * Conventions that the paper leaves open, and that the GPU path follows too
 * (written independently there), are stated next to the code that applies
 * them: the counter layout of the random stream, which uniform feeds which
 * draw, and the frame in which directions are built.
 *
 * Parity status of each function: see the pin list in the Python wrapper
 * (oracle/oracle.py).  The full (untruncated) porous-film effective
 * conductivity has no closed form: parity unpinned.  It is bounded by the
 * zero-radius (film) limit, the upper bound kappa_film (1 - porosity),
 * symmetry, the exact per-particle invariants, its first-event and
 * first-free-path truncations (pinned by quadrature) and the pore wall's
 * Lambertian law (pinned by the invariance of a uniform isotropic excess).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI 6.283185307179586
#define ORC_PI 3.141592653589793
#define ORC_HBAR 1.054571817e-34 /* J s (SI 2019 exact h / 2 pi) */
#define ORC_KB 1.380649e-23      /* J/K (SI 2019 exact)        */

/* ------------------------------------------------------------------------ */
/* Problem description (flat, ctypes friendly).                             */
/* ------------------------------------------------------------------------ */
enum { ORC_MAT_GRAY = 0, ORC_MAT_QUADRATIC = 1 };
enum { ORC_GEOM_PLANES = 0, ORC_GEOM_BULK = 1, ORC_GEOM_POROUS = 2 };
enum { ORC_WALL_BLACK = 0, ORC_WALL_DIFFUSE = 1, ORC_WALL_SPECULAR = 2, ORC_WALL_PARTIAL = 3 };
enum { ORC_SRC_WALLS = 0, ORC_SRC_GRADIENT = 1, ORC_SRC_PULSE = 2, ORC_SRC_INITIAL = 3 };
enum { ORC_FATE_ABSORBED = 0, ORC_FATE_MAX_SCATTER = 1, ORC_FATE_MAX_EVENTS = 2,
       ORC_FATE_T_FINAL = 3, ORC_FATE_MAX_COLLISIONS = 4 };

typedef struct {
    /* material */
    int32_t mat_kind;
    int32_t n_branch;
    int32_t n_bins_omega;
    int32_t pad0;
    double T_eq;
    double gray_v, gray_tau, gray_C;
    double c1[4], c2[4], degeneracy[4];
    double a_lattice, A, B, Cexp;
    double scatter_g;     /* mean cosine of the direction change at a relaxation
                             event: 0 isotropic (the paper's law), else the
                             Henyey-Greenstein law about the incoming direction */
    /* geometry */
    int32_t geom_kind;
    int32_t wall_lo, wall_hi, pore_wall;
    double L;             /* film / slab thickness along x [m]         */
    double pitch, radius; /* porous: square lattice in (y,z)           */
    int32_t cells_y, cells_z;
    /* PARTIAL walls: probability of a specular reflection at x = 0, x = L and
     * on the pores (the remainder is diffuse) */
    double spec_lo, spec_hi, spec_pore;
    /* source */
    int32_t src_kind;
    int32_t pad1;
    double dT_lo, dT_hi;  /* WALLS: T_wall - T_eq at x = 0 and x = L    */
    double dTdz;          /* GRADIENT                                   */
    double pulse_sigma_x, pulse_sigma_t, pulse_t_center, pulse_energy;
    double pulse_y0, pulse_z0;
    double init_dT;       /* INITIAL: T_i - T_eq inside init_x_lo < x < init_x_hi at t = 0 */
    double init_x_lo, init_x_hi;
    /* run */
    uint64_t n_particles;
    uint64_t seed;
    uint32_t instance_id;
    uint32_t max_scatter; /* terminate at this scattering event; 0 = no cap */
    uint32_t max_events;  /* terminate after this many segments (>= 1)    */
    uint32_t max_collisions; /* terminate at this many scatterings + wall
                                hits (periodic faces excluded); 0 = no cap */
    int32_t n_bins_x;     /* slab profile bins along x (0 = off)          */
    int32_t n_batch;      /* batch groups for the profile error bars      */
    int32_t grid_nx, grid_ny, grid_nz, n_samples;
    int32_t n_hj;         /* per-scattering-index flux tally length        */
    double t_final;       /* transient end time (0 = steady, infinite)     */
    double sample_dt;     /* transient sample spacing                      */
    int32_t n_threads;
    int32_t record_particles;
    /* POROUS, GRADIENT: steady maps over the (y, z) unit cell, integrated
     * through the thickness, map_ny x map_nz cells (0 = off); their error
     * bars come from the n_batch groups */
    int32_t map_ny, map_nz;
} orc_problem;

typedef struct {
    int8_t sign;
    int8_t fate;
    int16_t pad;
    uint32_t n_seg, n_scat, n_wall, n_periodic;
    uint32_t mode0;
    double L_axis;  /* algebraic length along the flux axis (x for WALLS, z else) */
    double x0, t0;  /* emission position along x and emission time              */
} orc_particle;

typedef struct {
    double P_total;     /* source power (W per m^2 of wall area for WALLS,
                           W per unit-cell volume normalisation otherwise)   */
    double E_eff_dot;   /* steady: effective power per particle              */
    double E_eff;       /* transient: energy per particle                    */
    double C_tot;       /* sum of C_b                                        */
    double sum_sL, sum_sL2;
    double flux, flux_se;   /* q along the flux axis [W/m^2]                 */
    double kappa, kappa_se; /* GRADIENT: -q/(dT/dz)                          */
    double kappa_solid;     /* porous: flux averaged over the solid only      */
    double psi, psi_se;     /* WALLS: q / (sum C v /4 * (dT_lo - dT_hi))      */
    uint64_t particles, segments, scatters, wall_hits, periodic, truncated, absorbed;
} orc_result;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror and   */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds  */
/* of two 32x32->64 multiplies on words 0 and 2 with a Weyl key schedule.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u; /* golden ratio      */
        k1 += 0xBB67AE85u; /* sqrt(3) - 1       */
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Four uniforms in ]0,1[ (step II requires R in ]0,1[): (r + 1/2) 2^-32.
 * Counter layout: (event, block, particle, instance); key = seed. */
static void draw4(const orc_problem* p, uint32_t event, uint32_t block, uint64_t pid,
                  double u[4])
{
    uint32_t ctr[4] = {event, block, (uint32_t)pid, p->instance_id};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = ((double)r[i] + 0.5) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Material: per-mode (omega_b, v_b, tau_b, C_b) at T_eq.                    */
/* C_b = g_p D_p(omega_b) hbar omega_b d f_BE/dT domega  (the paper's        */
/* D de^eq/dT summed over the bin; the 1/(4 pi) of C_{omega,p} is applied    */
/* in the angular integrals of the sources).                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    double* omega;
    double* v;
    double* tau;
    double* C;
    double* Lambda;
    double* cdf_emit; /* cumulative of C_b v_b  (boundary, gradient, pulse sources) */
    double* cdf_scat; /* cumulative of C_b / tau_b  (Eq. 2)                         */
    double* cdf_init; /* cumulative of C_b  (initial-condition source)               */
    double C_tot, Cv_sum;
} orc_mat;

static void mat_free(orc_mat* m)
{
    free(m->omega); free(m->v); free(m->tau); free(m->C); free(m->Lambda);
    free(m->cdf_emit); free(m->cdf_scat); free(m->cdf_init);
    memset(m, 0, sizeof(*m));
}

static int mat_alloc(orc_mat* m, int n)
{
    m->n = n;
    m->omega = calloc(n, sizeof(double));
    m->v = calloc(n, sizeof(double));
    m->tau = calloc(n, sizeof(double));
    m->C = calloc(n, sizeof(double));
    m->Lambda = calloc(n, sizeof(double));
    m->cdf_emit = calloc(n, sizeof(double));
    m->cdf_scat = calloc(n, sizeof(double));
    m->cdf_init = calloc(n, sizeof(double));
    return (m->omega && m->v && m->tau && m->C && m->Lambda && m->cdf_emit && m->cdf_scat && m->cdf_init) ? 0 : -1;
}

/* Isotropic dispersion omega(k) = c1 k + c2 k^2 per branch, n_bins equal-width
 * bins on [0, omega_max]; k_max = min(2 pi / a, c1 / (2 |c2|)) when c2 < 0 so
 * that the group velocity stays positive; relaxation time
 * 1/tau = A omega^4 + B omega^2 T exp(-C/T), the same law for every branch. */
static int mat_build(const orc_problem* p, orc_mat* m)
{
    if (p->mat_kind == ORC_MAT_GRAY) {
        if (mat_alloc(m, 1)) return -1;
        m->omega[0] = 0.0;
        m->v[0] = p->gray_v;
        m->tau[0] = p->gray_tau;
        m->C[0] = p->gray_C;
    } else if (p->mat_kind == ORC_MAT_QUADRATIC) {
        int nb = p->n_bins_omega;
        if (nb < 1 || p->n_branch < 1 || p->n_branch > 4) return -1;
        if (mat_alloc(m, nb * p->n_branch)) return -1;
        double T = p->T_eq;
        for (int br = 0; br < p->n_branch; ++br) {
            double c1 = p->c1[br], c2 = p->c2[br], g = p->degeneracy[br];
            double kmax = 2.0 * ORC_PI / p->a_lattice;
            if (c2 < 0.0 && c1 / (2.0 * fabs(c2)) < kmax) kmax = c1 / (2.0 * fabs(c2));
            double wmax = c1 * kmax + c2 * kmax * kmax;
            double dw = wmax / nb;
            for (int b = 0; b < nb; ++b) {
                int i = br * nb + b;
                double w = (b + 0.5) * dw;
                double vg = sqrt(c1 * c1 + 4.0 * c2 * w); /* d omega / dk      */
                double k = 2.0 * w / (c1 + vg);            /* root with vg > 0  */
                double dos = k * k / (2.0 * ORC_PI * ORC_PI * vg);
                double x = ORC_HBAR * w / (ORC_KB * T);
                double em1 = expm1(x);
                double dfdT = x * exp(x) / (em1 * em1 * T);
                m->omega[i] = w;
                m->v[i] = vg;
                m->C[i] = g * dos * ORC_HBAR * w * dfdT * dw;
                m->tau[i] = 1.0 / (p->A * w * w * w * w + p->B * w * w * T * exp(-p->Cexp / T));
            }
        }
    } else {
        return -1;
    }
    double ce = 0.0, cs = 0.0;
    m->C_tot = 0.0;
    m->Cv_sum = 0.0;
    for (int i = 0; i < m->n; ++i) {
        m->Lambda[i] = m->v[i] * m->tau[i];
        ce += m->C[i] * m->v[i];
        cs += m->C[i] / m->tau[i];
        m->cdf_emit[i] = ce;
        m->cdf_scat[i] = cs;
        m->cdf_init[i] = m->C_tot + m->C[i];
        m->C_tot += m->C[i];
    }
    m->Cv_sum = ce;
    return 0;
}

/* Inverse CDF: the first mode whose cumulative weight exceeds u * total. */
static int draw_mode(const double* cdf, int n, double u)
{
    double target = u * cdf[n - 1];
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Particle state and direction construction.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    double x, y, z;     /* position; y,z local to the unit cell for POROUS   */
    int64_t cy, cz;     /* POROUS: unwrapped unit-cell indices               */
    double ox, oy, oz;  /* unit direction Omega                              */
    int mode;
    int sign;
    double t;           /* internal time                                     */
} orc_state;

/* Direction with cosine mu about axis a in {0:x, 2:z} and azimuth phi about it.
 * Axis x: (mu, s cos phi, s sin phi).  Axis z: (s cos phi, s sin phi, mu).
 * s = sqrt(max(0, 1 - mu mu)). */
static void dir_axis(int axis, double mu, double u_phi, double* ox, double* oy, double* oz)
{
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    double phi = ORC_TWO_PI * u_phi;
    double c = cos(phi), sn = sin(phi);
    if (axis == 0) { *ox = mu; *oy = s * c; *oz = s * sn; }
    else { *ox = s * c; *oy = s * sn; *oz = mu; }
}

/* Anisotropic generalisation of the relaxation event's direction (the paper
 * uses an isotropic redraw and notes that other laws fit the same scheme):
 * the Henyey-Greenstein law with mean cosine g != 0 about the incoming
 * direction n.  The cosine mu = Omega'.n inverts the law's CDF
 * F(mu) = (1 - g^2)/(2g) [(1 + g^2 - 2 g mu)^(-1/2) - (1 + g)^(-1)] at u_mu;
 * the azimuth is 2 pi u_phi in the frame (b1, b2, n) of Duff et al.,
 * "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017. */
static void hg_direction(double g, double u_mu, double u_phi, double nx, double ny, double nz, double* ox,
                         double* oy, double* oz)
{
    double q = (1.0 - g * g) / (1.0 - g + 2.0 * g * u_mu);
    double mu = (1.0 + g * g - q * q) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    double phi = ORC_TWO_PI * u_phi;
    double c = cos(phi), sn = sin(phi);
    double sg = nz >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + nz);
    double b = nx * ny * a;
    double b1x = 1.0 + sg * nx * nx * a, b1y = sg * b, b1z = -sg * nx;
    double b2x = b, b2y = sg + ny * ny * a, b2z = -ny;
    *ox = mu * nx + s * (c * b1x + sn * b2x);
    *oy = mu * ny + s * (c * b1y + sn * b2y);
    *oz = mu * nz + s * (c * b1z + sn * b2z);
}

/* ------------------------------------------------------------------------ */
/* Thread-local tallies.                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double sum_sL, sum_sL2;
    uint64_t particles, segments, scatters, wall_hits, periodic, truncated, absorbed;
    double* T_sum;   /* [n_batch][n_bins_x] sum of s * time in bin          */
    double* q_sum;   /* [n_batch][n_bins_x] sum of s * x-displacement in bin */
    double* h_sum;   /* [n_hj] */
    double* h_sum2;  /* [n_hj] */
    int64_t* grid;   /* [n_samples][nz][ny][nx] signed counts                */
    double* mT_sum;  /* [n_batch][map_nz][map_ny] sum of s * time over the cell */
    double* mq_sum;  /* [n_batch][map_nz][map_ny] sum of s * z-displacement    */
} orc_tally;

static void tally_free(orc_tally* t)
{
    free(t->T_sum); free(t->q_sum); free(t->h_sum); free(t->h_sum2); free(t->grid);
    free(t->mT_sum); free(t->mq_sum);
    memset(t, 0, sizeof(*t));
}

static size_t grid_cells(const orc_problem* p)
{
    return (size_t)p->n_samples * p->grid_nz * p->grid_ny * p->grid_nx;
}

static size_t map_cells(const orc_problem* p)
{
    return (p->map_ny > 0 && p->map_nz > 0) ? (size_t)p->map_ny * p->map_nz : 0;
}

static int tally_alloc(const orc_problem* p, orc_tally* t)
{
    memset(t, 0, sizeof(*t));
    size_t nb = (size_t)(p->n_bins_x > 0 ? p->n_bins_x : 0) * (size_t)(p->n_batch > 0 ? p->n_batch : 1);
    if (nb) {
        t->T_sum = calloc(nb, sizeof(double));
        t->q_sum = calloc(nb, sizeof(double));
        if (!t->T_sum || !t->q_sum) return -1;
    }
    if (p->n_hj > 0) {
        t->h_sum = calloc(p->n_hj, sizeof(double));
        t->h_sum2 = calloc(p->n_hj, sizeof(double));
        if (!t->h_sum || !t->h_sum2) return -1;
    }
    if (p->n_samples > 0) {
        t->grid = calloc(grid_cells(p), sizeof(int64_t));
        if (!t->grid) return -1;
    }
    if (map_cells(p) > 0) {
        size_t nm = map_cells(p) * (size_t)(p->n_batch > 0 ? p->n_batch : 1);
        t->mT_sum = calloc(nm, sizeof(double));
        t->mq_sum = calloc(nm, sizeof(double));
        if (!t->mT_sum || !t->mq_sum) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Step I: initial state.                                                    */
/* Random layout: block 0 of event 0 gives (u0 source specific, u1 mode,     */
/* u2 polar cosine, u3 azimuth); rejection loops use blocks 1, 2, ... for    */
/* positions and blocks 65, 66, ... for pulse emission times.               */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_TRIES 64

static int in_pore(const orc_problem* p, double y, double z)
{
    if (p->radius <= 0.0) return 0;
    double dy = y - 0.5 * p->pitch, dz = z - 0.5 * p->pitch;
    return dy * dy + dz * dz < p->radius * p->radius;
}

static void emit(const orc_problem* p, const orc_mat* m, uint64_t pid, orc_state* s)
{
    double u[4];
    draw4(p, 0u, 0u, pid, u);
    memset(s, 0, sizeof(*s));
    s->mode = draw_mode(m->cdf_emit, m->n, u[1]);
    if (p->src_kind == ORC_SRC_WALLS) {
        /* Isothermal black walls: each wall emits V_g cos(theta) C |T_b - T_eq|
         * into the domain; the wall is picked in proportion to |T_b - T_eq|,
         * the sign is sgn(T_b - T_eq), the direction is cosine weighted. */
        double wlo = fabs(p->dT_lo), whi = fabs(p->dT_hi);
        int lo = u[0] * (wlo + whi) < wlo;
        double mu = sqrt(u[2]);
        dir_axis(0, mu, u[3], &s->ox, &s->oy, &s->oz);
        if (lo) { s->x = 0.0; s->sign = p->dT_lo >= 0.0 ? 1 : -1; }
        else { s->x = p->L; s->ox = -s->ox; s->sign = p->dT_hi >= 0.0 ? 1 : -1; }
        s->t = 0.0;
    } else if (p->src_kind == ORC_SRC_GRADIENT) {
        /* Eq. 6: volumetric source -D/(4 pi) V_g cos(theta) de/dT dT/dz.  Mode
         * weight C_b v_b, |cos theta| weighted about z, sign
         * sgn(-cos(theta) dT/dz); equal numbers of each sign: even particle
         * ids are positive, odd ids negative. */
        s->sign = (pid & 1u) ? -1 : 1;
        double amu = sqrt(u[2]);
        double dir_sign = (double)s->sign * (p->dTdz > 0.0 ? -1.0 : 1.0);
        dir_axis(2, dir_sign * amu, u[3], &s->ox, &s->oy, &s->oz);
        s->t = 0.0;
        if (p->geom_kind == ORC_GEOM_PLANES) {
            s->x = u[0] * p->L;
        } else if (p->geom_kind == ORC_GEOM_BULK) {
            s->x = 0.0;
        } else { /* POROUS: uniform in the solid part of the periodic domain */
            s->x = u[0] * p->L;
            for (uint32_t b = 1; b <= ORC_MAX_TRIES; ++b) {
                double v[4];
                draw4(p, 0u, b, pid, v);
                double Y = v[0] * p->pitch * p->cells_y;
                double Z = v[1] * p->pitch * p->cells_z;
                int64_t cy = (int64_t)floor(Y / p->pitch), cz = (int64_t)floor(Z / p->pitch);
                if (cy >= p->cells_y) cy = p->cells_y - 1;
                if (cz >= p->cells_z) cz = p->cells_z - 1;
                double yl = Y - cy * p->pitch, zl = Z - cz * p->pitch;
                s->cy = cy; s->cz = cz; s->y = yl; s->z = zl;
                if (!in_pore(p, yl, zl)) break;
            }
        }
    } else if (p->src_kind == ORC_SRC_INITIAL) {
        /* Initial condition C_{w,p} |T_i - T_eq| delta(t) (text after the
         * algorithm): at t = 0, uniform in the region init_x_lo < x <
         * init_x_hi (solid part), mode weight C_b, isotropic direction, sign
         * sgn(T_i - T_eq).  u1 mode, u2 polar cosine (2u - 1 about z), u3
         * azimuth; blocks 1.. the lateral position as for the gradient source. */
        s->mode = draw_mode(m->cdf_init, m->n, u[1]);
        s->sign = p->init_dT >= 0.0 ? 1 : -1;
        s->x = p->init_x_lo + u[0] * (p->init_x_hi - p->init_x_lo);
        dir_axis(2, 2.0 * u[2] - 1.0, u[3], &s->ox, &s->oy, &s->oz);
        s->t = 0.0;
        for (uint32_t b = 1; b <= ORC_MAX_TRIES; ++b) {
            double v[4];
            draw4(p, 0u, b, pid, v);
            double Y = v[0] * p->pitch * p->cells_y;
            double Z = v[1] * p->pitch * p->cells_z;
            int64_t cy = (int64_t)floor(Y / p->pitch), cz = (int64_t)floor(Z / p->pitch);
            if (cy >= p->cells_y) cy = p->cells_y - 1;
            if (cz >= p->cells_z) cz = p->cells_z - 1;
            double yl = Y - cy * p->pitch, zl = Z - cz * p->pitch;
            s->cy = cy; s->cz = cz; s->y = yl; s->z = zl;
            if (!in_pore(p, yl, zl)) break;
        }
    } else { /* ORC_SRC_PULSE: surface heat pulse on the top face x = L */
        s->sign = 1;
        s->x = p->L;
        double mu = sqrt(u[2]);
        dir_axis(0, mu, u[3], &s->ox, &s->oy, &s->oz);
        s->ox = -s->ox; /* into the film */
        double Dy = p->pitch * p->cells_y, Dz = p->pitch * p->cells_z;
        for (uint32_t b = 1; b <= ORC_MAX_TRIES; ++b) {
            double v[4];
            draw4(p, 0u, b, pid, v);
            double r = p->pulse_sigma_x * sqrt(-2.0 * log(v[0]));
            double Y = p->pulse_y0 + r * cos(ORC_TWO_PI * v[1]);
            double Z = p->pulse_z0 + r * sin(ORC_TWO_PI * v[1]);
            Y -= Dy * floor(Y / Dy);
            Z -= Dz * floor(Z / Dz);
            int64_t cy = (int64_t)floor(Y / p->pitch), cz = (int64_t)floor(Z / p->pitch);
            if (cy >= p->cells_y) cy = p->cells_y - 1;
            if (cz >= p->cells_z) cz = p->cells_z - 1;
            if (cy < 0) cy = 0;
            if (cz < 0) cz = 0;
            s->cy = cy; s->cz = cz;
            s->y = Y - cy * p->pitch;
            s->z = Z - cz * p->pitch;
            if (!in_pore(p, s->y, s->z)) break;
        }
        s->t = p->pulse_t_center;
        for (uint32_t b = 65; b < 65 + ORC_MAX_TRIES; ++b) {
            double v[4];
            draw4(p, 0u, b, pid, v);
            double t0 = p->pulse_t_center + p->pulse_sigma_t * sqrt(-2.0 * log(v[0])) * cos(ORC_TWO_PI * v[1]);
            if (t0 >= 0.0) { s->t = t0; break; }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Step III: first boundary along the ray (distance along the unit direction).*/
/* ------------------------------------------------------------------------ */
enum { HIT_NONE = 0, HIT_XLO, HIT_XHI, HIT_CYL, HIT_YLO, HIT_YHI, HIT_ZLO, HIT_ZHI };

static double first_boundary(const orc_problem* p, const orc_state* s, int* kind)
{
    double best = INFINITY;
    *kind = HIT_NONE;
    if (p->geom_kind == ORC_GEOM_BULK) return best;
    /* film / slab walls at x = 0 and x = L */
    if (s->ox > 0.0) { best = (p->L - s->x) / s->ox; *kind = HIT_XHI; }
    else if (s->ox < 0.0) { best = -s->x / s->ox; *kind = HIT_XLO; }
    if (p->geom_kind != ORC_GEOM_POROUS) return best;
    /* cylindrical pore along x through the cell centre */
    if (p->radius > 0.0) {
        double ry = s->y - 0.5 * p->pitch, rz = s->z - 0.5 * p->pitch;
        double a = s->oy * s->oy + s->oz * s->oz;
        double b = ry * s->oy + rz * s->oz;
        double c = ry * ry + rz * rz - p->radius * p->radius;
        if (a > 0.0 && b < 0.0) {
            double disc = b * b - a * c;
            if (disc >= 0.0) {
                double t = c / (-b + sqrt(disc));
                if (t < 0.0) t = 0.0;
                if (t < best) { best = t; *kind = HIT_CYL; }
            }
        }
    }
    /* unit-cell faces in y and z (periodic) */
    if (s->oy > 0.0) { double t = (p->pitch - s->y) / s->oy; if (t < best) { best = t; *kind = HIT_YHI; } }
    else if (s->oy < 0.0) { double t = -s->y / s->oy; if (t < best) { best = t; *kind = HIT_YLO; } }
    if (s->oz > 0.0) { double t = (p->pitch - s->z) / s->oz; if (t < best) { best = t; *kind = HIT_ZHI; } }
    else if (s->oz < 0.0) { double t = -s->z / s->oz; if (t < best) { best = t; *kind = HIT_ZLO; } }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Step V: sample the contribution of a segment.                             */
/* ------------------------------------------------------------------------ */
/* Slab profiles along x (Eq. 4 per bin): the time a segment spends in each
 * bin, and the displacement it makes there along the flux axis -- x for the
 * walls source, z for the gradient source (the in-plane flux of a film by
 * depth: the z displacement over an x-length len is len |oz / ox|, signed by
 * oz).  Batch groups: particle ids mod n_batch, or particle pairs (2i, 2i + 1)
 * for the gradient source, whose even and odd ids carry opposite signs. */
static void tally_slab_bins(const orc_problem* p, const orc_mat* m, orc_tally* tl, uint64_t pid,
                            int sign, double xa, double xb, double ox, double oz, double seg, double dt_seg,
                            int mode)
{
    const int grad = p->src_kind == ORC_SRC_GRADIENT;
    int nb = p->n_bins_x;
    double dx = p->L / nb;
    uint64_t B = (uint64_t)(p->n_batch > 0 ? p->n_batch : 1);
    int g = (int)((grad ? pid >> 1 : pid) % B);
    double* T = tl->T_sum + (size_t)g * nb;
    double* q = tl->q_sum + (size_t)g * nb;
    double lo = fmin(xa, xb), hi = fmax(xa, xb);
    int k0 = (int)floor(lo / dx), k1 = (int)floor(hi / dx);
    if (k0 < 0) k0 = 0;
    if (k1 > nb - 1) k1 = nb - 1;
    if (k0 > nb - 1) k0 = nb - 1;
    if (k1 < 0) k1 = 0;
    if (ox == 0.0) { /* a flight parallel to the walls stays in one bin */
        T[k0] += sign * dt_seg;
        if (grad) q[k0] += sign * (oz * seg);
        return;
    }
    double speed_x = m->v[mode] * fabs(ox);
    for (int k = k0; k <= k1; ++k) {
        double a = fmax(lo, k * dx), b = fmin(hi, (k + 1) * dx);
        if (k == nb - 1) b = hi;
        if (k == 0) a = lo;
        double len = b - a;
        if (len <= 0.0) continue;
        T[k] += sign * (len / speed_x);
        if (grad)
            q[k] += sign * (len * oz / fabs(ox));
        else
            q[k] += sign * (ox > 0.0 ? len : -len);
    }
}

/* Clip the parameter interval [*a, *b] of the line x0 + d t to lo <= x < hi
 * (lo <= x <= hi when `last`, the top cell of the range). */
static void clip_axis(double x0, double d, double lo, double hi, int last, double* a, double* b)
{
    if (d == 0.0) {
        int inside = x0 >= lo && (last ? x0 <= hi : x0 < hi);
        if (!inside) *b = *a - 1.0;
        return;
    }
    double t1 = (lo - x0) / d, t2 = (hi - x0) / d;
    if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; }
    if (t1 > *a) *a = t1;
    if (t2 < *b) *b = t2;
}

/* Steady maps (Eq. 4 per map cell): over the (y, z) unit cell, integrated
 * through the thickness, a segment adds s * (the time it spends over the
 * cell) to the cell's temperature sum and s * (its z displacement over the
 * cell) to its flux sum.  The segment [0, seg] of the ray (y, z) + (oy, oz) t
 * is clipped to each cell's y and z extents in turn; cells outside the
 * segment's bounding box cannot meet it and are skipped. */
static void tally_map(const orc_problem* p, const orc_mat* m, orc_tally* tl, uint64_t pid, const orc_state* s,
                      double seg)
{
    const int ny = p->map_ny, nz = p->map_nz;
    const double dy = p->pitch / ny, dz = p->pitch / nz;
    const size_t cells = (size_t)ny * nz;
    /* batch group of the particle pair (2i, 2i + 1): the gradient source
     * gives even ids one sign and odd ids the other, so a group must hold
     * pairs for its estimate to see both signs */
    const int g = (int)((pid >> 1) % (uint64_t)(p->n_batch > 0 ? p->n_batch : 1));
    double* T = tl->mT_sum + (size_t)g * cells;
    double* q = tl->mq_sum + (size_t)g * cells;
    const double y1 = s->y + s->oy * seg, z1 = s->z + s->oz * seg;
    int j0 = (int)floor(fmin(s->y, y1) / dy), j1 = (int)floor(fmax(s->y, y1) / dy);
    int k0 = (int)floor(fmin(s->z, z1) / dz), k1 = (int)floor(fmax(s->z, z1) / dz);
    if (j0 < 0) j0 = 0;
    if (k0 < 0) k0 = 0;
    if (j1 > ny - 1) j1 = ny - 1;
    if (k1 > nz - 1) k1 = nz - 1;
    const double vg = m->v[s->mode];
    for (int k = k0; k <= k1; ++k)
        for (int j = j0; j <= j1; ++j) {
            double a = 0.0, b = seg;
            clip_axis(s->y, s->oy, j * dy, (j + 1) * dy, j == ny - 1, &a, &b);
            clip_axis(s->z, s->oz, k * dz, (k + 1) * dz, k == nz - 1, &a, &b);
            if (b <= a) continue;
            T[(size_t)k * ny + j] += s->sign * ((b - a) / vg);
            q[(size_t)k * ny + j] += s->sign * (s->oz * (b - a));
        }
}

/* Solid area of the map cell [ya, yb] x [za, zb] of the unit cell: the cell
 * minus its overlap with the pore disk (centre (c, c), radius r).  The overlap
 * is the integral over y of the z-length shared by [za, zb] and the disk's
 * chord; with y = c + r sin(theta) the chord half-length is r cos(theta) and
 * the integrand is smooth between the angles where the chord's ends cross za
 * or zb, so each such piece is integrated by 20-point Gauss-Legendre. */
static double chord_overlap(double c, double r, double za, double zb, double th)
{
    const double h = r * cos(th);
    double lo = fmax(za, c - h), hi = fmin(zb, c + h);
    return hi > lo ? (hi - lo) * r * cos(th) : 0.0;
}

/* Positive nodes and weights of 20-point Gauss-Legendre quadrature on
 * [-1, 1]: Newton's method on the Legendre polynomial P_20 (three-term
 * recurrence), started from the Chebyshev-like guess cos(pi (i - 1/4) / 20.5). */
static void gauss_legendre20(double* x, double* w)
{
    const int n = 20;
    for (int i = 1; i <= n / 2; ++i) {
        double z = cos(ORC_PI * (i - 0.25) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i - 1] = z;
        w[i - 1] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static double map_cell_solid(double c, double r, double ya, double yb, double za, double zb)
{
    const double full = (yb - ya) * (zb - za);
    if (r <= 0.0) return full;
    double lo = fmax(ya, c - r), hi = fmin(yb, c + r);
    if (hi <= lo) return full;
    double t_lo = asin(fmax(-1.0, fmin(1.0, (lo - c) / r)));
    double t_hi = asin(fmax(-1.0, fmin(1.0, (hi - c) / r)));
    /* breakpoints: c + r cos(th) = zb or za, c - r cos(th) = za or zb */
    double brk[10];
    int nb = 0;
    brk[nb++] = t_lo;
    const double zs[2] = {za, zb};
    for (int i = 0; i < 2; ++i) {
        double w = fabs(zs[i] - c) / r;
        if (w < 1.0) {
            double a = acos(w);
            if (a > t_lo && a < t_hi) brk[nb++] = a;
            if (-a > t_lo && -a < t_hi) brk[nb++] = -a;
        }
    }
    brk[nb++] = t_hi;
    for (int i = 1; i < nb; ++i) /* insertion sort */
        for (int j = i; j > 0 && brk[j] < brk[j - 1]; --j) { double t = brk[j]; brk[j] = brk[j - 1]; brk[j - 1] = t; }
    double x20[10], w20[10];
    gauss_legendre20(x20, w20);
    double overlap = 0.0;
    for (int i = 0; i + 1 < nb; ++i) {
        double a = brk[i], b = brk[i + 1], mid = 0.5 * (a + b), half = 0.5 * (b - a);
        if (half <= 0.0) continue;
        double sum = 0.0;
        for (int k = 0; k < 10; ++k)
            sum += w20[k] * (chord_overlap(c, r, za, zb, mid - half * x20[k]) +
                             chord_overlap(c, r, za, zb, mid + half * x20[k]));
        overlap += half * sum;
    }
    return full - overlap;
}

static int grid_index(double v, double extent, int n)
{
    int i = (int)floor(v / extent * n);
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    return i;
}

/* Eq. 3: at every sample time t'_k in [t_a, t_b) the particle adds its sign
 * to the cell that holds its (linearly interpolated) position. */
static void tally_transient(const orc_problem* p, const orc_mat* m, orc_tally* tl, const orc_state* s,
                            double t_a, double t_b)
{
    double dts = p->sample_dt;
    double t_end = t_b < p->t_final ? t_b : p->t_final;
    /* the rounded quotient can land one past the first t'_k >= t_a; start one
     * early and let the exact comparisons below decide */
    long k = (long)ceil(t_a / dts - 0.5) - 1;
    if (k < 0) k = 0;
    double Dy = p->pitch * p->cells_y, Dz = p->pitch * p->cells_z;
    double vg = m->v[s->mode];
    for (; k < p->n_samples; ++k) {
        double ts = (k + 0.5) * dts;
        if (ts < t_a) continue;
        if (ts >= t_b || ts > t_end) break;
        double d = vg * (ts - t_a);
        double x = s->x + s->ox * d;
        double y = s->y + s->oy * d;
        double z = s->z + s->oz * d;
        int64_t cy = s->cy % p->cells_y; if (cy < 0) cy += p->cells_y;
        int64_t cz = s->cz % p->cells_z; if (cz < 0) cz += p->cells_z;
        double Y = cy * p->pitch + y, Z = cz * p->pitch + z;
        int ix = grid_index(x, p->L, p->grid_nx);
        int iy = grid_index(Y, Dy, p->grid_ny);
        int iz = grid_index(Z, Dz, p->grid_nz);
        size_t cell = (((size_t)k * p->grid_nz + iz) * p->grid_ny + iy) * p->grid_nx + ix;
        tl->grid[cell] += s->sign;
    }
}

/* ------------------------------------------------------------------------ */
/* Steps I-VI for one particle.                                              */
/* ------------------------------------------------------------------------ */
static void trace_particle(const orc_problem* p, const orc_mat* m, uint64_t pid, orc_tally* tl,
                           orc_particle* rec)
{
    orc_state s;
    emit(p, m, pid, &s); /* step I */
    const int transient = p->t_final > 0.0;
    const int axis_x = p->src_kind == ORC_SRC_WALLS;
    double x_emit = s.x, t_emit = s.t;
    int mode0 = s.mode;
    uint32_t n_seg = 0, n_scat = 0, n_wall = 0, n_per = 0;
    double L_axis = 0.0; /* algebraic length along the flux axis (after Eq. 4) */
    double h_run = 0.0;  /* flux-axis length since the last scattering event    */
    int fate = ORC_FATE_MAX_EVENTS;
    for (uint32_t k = 1;; ++k) {
        double u[4];
        draw4(p, k, 0u, pid, u);
        /* step II: flight time to the next relaxation event */
        double tau = m->tau[s.mode];
        double vg = m->v[s.mode];
        double dt = -tau * log(u[0]);
        /* step III: boundary search during dt */
        int kind;
        double d_b = first_boundary(p, &s, &kind);
        double dist = m->Lambda[s.mode] * -log(u[0]); /* = |V_g| dt */
        int hit = kind != HIT_NONE && d_b <= dist;
        double seg = hit ? d_b : dist;
        double dt_seg = hit ? d_b / vg : dt;
        double xa = s.x, t_a = s.t;
        double dz = s.oz * seg, dxs = s.ox * seg;
        /* step V: contribution of the segment [x_0, x_new] */
        if (transient) tally_transient(p, m, tl, &s, t_a, t_a + dt_seg);
        double x_new = s.x + dxs;
        if (hit && kind == HIT_XLO) x_new = 0.0;
        if (hit && kind == HIT_XHI) x_new = p->L;
        if (p->n_bins_x > 0) tally_slab_bins(p, m, tl, pid, s.sign, xa, x_new, s.ox, s.oz, seg, dt_seg, s.mode);
        if (map_cells(p) > 0) tally_map(p, m, tl, pid, &s, seg);
        double dL = axis_x ? (x_new - xa) : dz;
        L_axis += dL;
        h_run += dL;
        /* advance position and time (steps IVa / IVb) */
        s.x = x_new;
        s.y += s.oy * seg;
        s.z += dz;
        s.t = t_a + dt_seg;
        ++n_seg;
        int absorbed = 0;
        if (hit) {
            int wall_type = -1;
            double spec = 0.0;
            if (kind == HIT_XLO) { wall_type = p->wall_lo; spec = p->spec_lo; }
            else if (kind == HIT_XHI) { wall_type = p->wall_hi; spec = p->spec_hi; }
            else if (kind == HIT_CYL) { wall_type = p->pore_wall; spec = p->spec_pore; }
            /* partially specular wall: specular with probability spec, else
             * diffuse; the draw is the flight's second uniform, which only a
             * relaxation event uses otherwise */
            if (wall_type == ORC_WALL_PARTIAL) wall_type = u[1] < spec ? ORC_WALL_SPECULAR : ORC_WALL_DIFFUSE;
            if (wall_type >= 0) {
                ++n_wall;
                if (wall_type == ORC_WALL_BLACK) {
                    absorbed = 1;
                } else if (kind == HIT_XLO || kind == HIT_XHI) {
                    if (wall_type == ORC_WALL_SPECULAR) s.ox = -s.ox;
                    else { /* diffuse: Lambertian about the inward normal */
                        dir_axis(0, sqrt(u[2]), u[3], &s.ox, &s.oy, &s.oz);
                        if (kind == HIT_XHI) s.ox = -s.ox;
                    }
                } else { /* pore wall: normal from the axis to the hit point */
                    double ny = (s.y - 0.5 * p->pitch) / p->radius;
                    double nz = (s.z - 0.5 * p->pitch) / p->radius;
                    if (wall_type == ORC_WALL_SPECULAR) {
                        double dn = s.oy * ny + s.oz * nz;
                        s.oy -= 2.0 * dn * ny;
                        s.oz -= 2.0 * dn * nz;
                    } else {
                        double mu = sqrt(u[2]);
                        double st = sqrt(fmax(0.0, 1.0 - mu * mu));
                        double phi = ORC_TWO_PI * u[3];
                        double c = cos(phi), sn = sin(phi);
                        s.ox = st * c;
                        s.oy = mu * ny - st * sn * nz;
                        s.oz = mu * nz + st * sn * ny;
                    }
                }
            } else { /* periodic unit-cell face: reinsert on the opposite face */
                ++n_per;
                if (kind == HIT_YHI) { s.y = 0.0; s.cy += 1; }
                else if (kind == HIT_YLO) { s.y = p->pitch; s.cy -= 1; }
                else if (kind == HIT_ZHI) { s.z = 0.0; s.cz += 1; }
                else if (kind == HIT_ZLO) { s.z = p->pitch; s.cz -= 1; }
            }
        } else {
            /* step IVb: relaxation event; (omega, p) from the normalised
             * Eq. 2, isotropic direction, sign kept */
            ++n_scat;
            if (p->n_hj > 0 && n_scat - 1 < (uint32_t)p->n_hj) {
                tl->h_sum[n_scat - 1] += s.sign * h_run;
                tl->h_sum2[n_scat - 1] += h_run * h_run;
            }
            h_run = 0.0;
            double in_x = s.ox, in_y = s.oy, in_z = s.oz;
            s.mode = draw_mode(m->cdf_scat, m->n, u[1]);
            dir_axis(2, 2.0 * u[2] - 1.0, u[3], &s.ox, &s.oy, &s.oz);
            if (p->scatter_g != 0.0) hg_direction(p->scatter_g, u[2], u[3], in_x, in_y, in_z, &s.ox, &s.oy, &s.oz);
        }
        /* step VI and the truncation rules */
        if (absorbed) { fate = ORC_FATE_ABSORBED; break; }
        if (transient && s.t > p->t_final) { fate = ORC_FATE_T_FINAL; break; }
        if (p->max_scatter > 0 && n_scat >= p->max_scatter) { fate = ORC_FATE_MAX_SCATTER; break; }
        /* first-free-path style truncation: a collision is a relaxation or a
         * wall / pore hit, not a crossing of a periodic unit-cell face */
        if (p->max_collisions > 0 && n_scat + n_wall >= p->max_collisions) { fate = ORC_FATE_MAX_COLLISIONS; break; }
        if (n_seg >= p->max_events) { fate = ORC_FATE_MAX_EVENTS; break; }
    }
    if (p->n_hj > 0 && n_scat < (uint32_t)p->n_hj && h_run != 0.0) {
        tl->h_sum[n_scat] += s.sign * h_run;
        tl->h_sum2[n_scat] += h_run * h_run;
    }
    double sL = s.sign * L_axis;
    tl->sum_sL += sL;
    tl->sum_sL2 += sL * sL;
    tl->particles += 1;
    tl->segments += n_seg;
    tl->scatters += n_scat;
    tl->wall_hits += n_wall;
    tl->periodic += n_per;
    if (fate == ORC_FATE_ABSORBED) tl->absorbed += 1;
    if (fate == ORC_FATE_MAX_SCATTER || fate == ORC_FATE_MAX_EVENTS || fate == ORC_FATE_MAX_COLLISIONS) tl->truncated += 1;
    if (rec) {
        rec->sign = (int8_t)s.sign;
        rec->fate = (int8_t)fate;
        rec->n_seg = n_seg;
        rec->n_scat = n_scat;
        rec->n_wall = n_wall;
        rec->n_periodic = n_per;
        rec->mode0 = (uint32_t)mode0;
        rec->L_axis = L_axis;
        rec->x0 = x_emit;
        rec->t0 = t_emit;
    }
}

/* ------------------------------------------------------------------------ */
/* Driver: disjoint particle ranges on host threads.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_problem* p;
    const orc_mat* m;
    uint64_t begin, end;
    orc_tally tally;
    orc_particle* records;
    int err;
} orc_job;

static void* run_job(void* arg)
{
    orc_job* j = (orc_job*)arg;
    for (uint64_t i = j->begin; i < j->end; ++i)
        trace_particle(j->p, j->m, i, &j->tally, j->records ? &j->records[i] : NULL);
    return NULL;
}

static int validate(const orc_problem* p)
{
    if (p->max_events < 1) return -1;
    if (p->geom_kind < 0 || p->geom_kind > 2) return -1;
    if (p->src_kind < 0 || p->src_kind > 3) return -1;
    if (p->geom_kind != ORC_GEOM_BULK && !(p->L > 0.0)) return -1;
    if (p->src_kind == ORC_SRC_WALLS && p->geom_kind != ORC_GEOM_PLANES) return -1;
    if (p->src_kind == ORC_SRC_PULSE && p->geom_kind != ORC_GEOM_POROUS) return -1;
    if (p->src_kind == ORC_SRC_INITIAL &&
        (p->geom_kind != ORC_GEOM_POROUS || !(p->t_final > 0.0) || p->init_dT == 0.0 ||
         !(p->init_x_lo >= 0.0) || !(p->init_x_hi <= p->L) || !(p->init_x_hi > p->init_x_lo)))
        return -1;
    if (p->geom_kind == ORC_GEOM_POROUS &&
        (!(p->pitch > 0.0) || p->radius < 0.0 || 2.0 * p->radius >= p->pitch || p->cells_y < 1 || p->cells_z < 1))
        return -1;
    if (p->n_bins_x > 0 && p->geom_kind != ORC_GEOM_PLANES) return -1;
    if (p->map_ny < 0 || p->map_nz < 0) return -1;
    if (map_cells(p) > 0 && (p->geom_kind != ORC_GEOM_POROUS || p->src_kind != ORC_SRC_GRADIENT || p->n_batch < 1))
        return -1;
    if (p->n_samples > 0 && (p->geom_kind != ORC_GEOM_POROUS || !(p->t_final > 0.0) || !(p->sample_dt > 0.0) ||
                             p->grid_nx < 1 || p->grid_ny < 1 || p->grid_nz < 1))
        return -1;
    if (p->n_particles > 0xFFFFFFFFull) return -1;
    if (p->wall_lo < 0 || p->wall_lo > 3 || p->wall_hi < 0 || p->wall_hi > 3) return -1;
    if (p->pore_wall < 1 || p->pore_wall > 3) return -1;
    if (!(p->scatter_g > -1.0 && p->scatter_g < 1.0)) return -1;
    if (!(p->spec_lo >= 0.0 && p->spec_lo <= 1.0) || !(p->spec_hi >= 0.0 && p->spec_hi <= 1.0) ||
        !(p->spec_pore >= 0.0 && p->spec_pore <= 1.0))
        return -1;
    return 0;
}

/* Output arrays (any may be NULL):
 *   T_mean/T_se [n_bins_x]   slab temperature T - T_eq (energy temperature)
 *   q_mean/q_se [n_bins_x]   slab heat flux per bin
 *   h_mean/h_se [n_hj]       flux contribution between scattering j and j+1
 *   grid_counts  [n_samples*nz*ny*nx] signed particle counts (Eq. 3)
 *   records [n_particles]    per-particle records
 *   maps [5][map_nz][map_ny] steady maps over the unit cell: T - T_eq(z)
 *                            over the solid of each map cell, its standard
 *                            error, the local z flux over that solid, its
 *                            standard error, and the cell's solid fraction
 *                            (NaN values where a cell holds no solid)     */
int orc_run(const orc_problem* p, orc_result* res, double* T_mean, double* T_se, double* q_mean,
            double* q_se, double* h_mean, double* h_se, int64_t* grid_counts, orc_particle* records,
            double* maps)
{
    if (validate(p)) return -1;
    orc_mat m;
    memset(&m, 0, sizeof(m));
    if (mat_build(p, &m)) { mat_free(&m); return -2; }
    int nt = p->n_threads > 0 ? p->n_threads : 1;
    uint64_t N = p->n_particles;
    if ((uint64_t)nt > N && N > 0) nt = (int)N;
    if (nt < 1) nt = 1;
    orc_job* jobs = calloc(nt, sizeof(orc_job));
    pthread_t* th = calloc(nt, sizeof(pthread_t));
    int rc = 0;
    for (int i = 0; i < nt; ++i) {
        jobs[i].p = p;
        jobs[i].m = &m;
        jobs[i].begin = N * (uint64_t)i / nt;
        jobs[i].end = N * (uint64_t)(i + 1) / nt;
        jobs[i].records = p->record_particles ? records : NULL;
        if (tally_alloc(p, &jobs[i].tally)) rc = -2;
    }
    if (rc == 0) {
        for (int i = 1; i < nt; ++i) pthread_create(&th[i], NULL, run_job, &jobs[i]);
        run_job(&jobs[0]);
        for (int i = 1; i < nt; ++i) pthread_join(th[i], NULL);
    }
    /* merge in thread order */
    orc_tally tot;
    memset(&tot, 0, sizeof(tot));
    if (rc == 0 && tally_alloc(p, &tot)) rc = -2;
    if (rc == 0) {
        size_t nb = (size_t)(p->n_bins_x > 0 ? p->n_bins_x : 0) * (size_t)(p->n_batch > 0 ? p->n_batch : 1);
        for (int i = 0; i < nt; ++i) {
            orc_tally* t = &jobs[i].tally;
            tot.sum_sL += t->sum_sL;
            tot.sum_sL2 += t->sum_sL2;
            tot.particles += t->particles;
            tot.segments += t->segments;
            tot.scatters += t->scatters;
            tot.wall_hits += t->wall_hits;
            tot.periodic += t->periodic;
            tot.truncated += t->truncated;
            tot.absorbed += t->absorbed;
            for (size_t b = 0; b < nb; ++b) { tot.T_sum[b] += t->T_sum[b]; tot.q_sum[b] += t->q_sum[b]; }
            for (int j = 0; j < p->n_hj; ++j) { tot.h_sum[j] += t->h_sum[j]; tot.h_sum2[j] += t->h_sum2[j]; }
            if (p->n_samples > 0)
                for (size_t c = 0; c < grid_cells(p); ++c) tot.grid[c] += t->grid[c];
            for (size_t c = 0; c < map_cells(p) * (size_t)(p->n_batch > 0 ? p->n_batch : 1); ++c) {
                tot.mT_sum[c] += t->mT_sum[c];
                tot.mq_sum[c] += t->mq_sum[c];
            }
        }
    }
    if (rc == 0) {
        /* Normalisation: N = deviational energy / E_eff (text after the
         * algorithm); steady runs use E_eff_dot = P / N (Eq. 4). */
        memset(res, 0, sizeof(*res));
        double Nd = (double)(N > 0 ? N : 1);
        double P = 0.0, Vref = 1.0, Vsolid = 1.0;
        if (p->src_kind == ORC_SRC_WALLS) {
            /* per unit wall area: each wall emits (1/4) sum_b C_b v_b |dT| */
            P = 0.25 * m.Cv_sum * (fabs(p->dT_lo) + fabs(p->dT_hi));
            Vref = p->L; /* flux averaged over the slab: divide by L */
        } else if (p->src_kind == ORC_SRC_GRADIENT) {
            if (p->geom_kind == ORC_GEOM_POROUS) {
                double cell = p->pitch * p->pitch * p->cells_y * p->cells_z;
                double pore = ORC_PI * p->radius * p->radius * p->cells_y * p->cells_z;
                Vsolid = (cell - pore) * p->L;
                Vref = cell * p->L;
            } else if (p->geom_kind == ORC_GEOM_PLANES) {
                Vsolid = p->L; Vref = p->L; /* per unit area in (y,z) */
            } else { Vsolid = 1.0; Vref = 1.0; }
            P = 0.5 * fabs(p->dTdz) * m.Cv_sum * Vsolid;
        } else {
            P = 0.0;
        }
        res->P_total = P;
        res->E_eff_dot = P / Nd;
        res->E_eff = p->src_kind == ORC_SRC_PULSE ? p->pulse_energy / Nd : 0.0;
        if (p->src_kind == ORC_SRC_INITIAL) {
            /* deviational energy of the initial condition: C_tot |T_i - T_eq| V */
            double area = (p->pitch * p->pitch - ORC_PI * p->radius * p->radius) * p->cells_y * p->cells_z;
            res->E_eff = m.C_tot * fabs(p->init_dT) * (p->init_x_hi - p->init_x_lo) * area / Nd;
        }
        res->C_tot = m.C_tot;
        res->sum_sL = tot.sum_sL;
        res->sum_sL2 = tot.sum_sL2;
        double mean = tot.sum_sL / Nd;
        double var = N > 1 ? (tot.sum_sL2 - Nd * mean * mean) / (Nd - 1.0) : 0.0;
        if (var < 0.0) var = 0.0;
        double se = sqrt(var / Nd);
        double scale = P / Vref; /* flux = E_eff_dot * sum(s L) / Vref */
        res->flux = scale * mean;
        res->flux_se = scale * se;
        if (p->src_kind == ORC_SRC_GRADIENT && p->dTdz != 0.0) {
            res->kappa = -res->flux / p->dTdz;
            res->kappa_se = res->flux_se / fabs(p->dTdz);
            res->kappa_solid = res->kappa * Vref / Vsolid;
        }
        if (p->src_kind == ORC_SRC_WALLS && p->dT_lo != p->dT_hi) {
            double denom = 0.25 * m.Cv_sum * (p->dT_lo - p->dT_hi);
            res->psi = res->flux / denom;
            res->psi_se = res->flux_se / fabs(denom);
        }
        res->particles = tot.particles;
        res->segments = tot.segments;
        res->scatters = tot.scatters;
        res->wall_hits = tot.wall_hits;
        res->periodic = tot.periodic;
        res->truncated = tot.truncated;
        res->absorbed = tot.absorbed;
        /* slab profiles: batch means over the n_batch groups */
        if (p->n_bins_x > 0) {
            int nb = p->n_bins_x, B = p->n_batch > 0 ? p->n_batch : 1;
            double dx = p->L / nb;
            for (int k = 0; k < nb; ++k) {
                double sT = 0, sT2 = 0, sq = 0, sq2 = 0;
                for (int g = 0; g < B; ++g) {
                    /* group g holds the particles with id = g mod B, or (gradient
                     * source) the particle pairs (2q, 2q + 1) with q = g mod B */
                    double ng = 0.0;
                    if (p->src_kind == ORC_SRC_GRADIENT) {
                        for (uint64_t e = 0; e < 2; ++e) {
                            uint64_t Q = N > e ? (N - e + 1) / 2 : 0;
                            ng += (double)(Q / B + ((uint64_t)g < Q % B ? 1 : 0));
                        }
                    } else {
                        ng = (double)(N / B + ((uint64_t)g < N % B ? 1 : 0));
                    }
                    if (ng <= 0) ng = 1;
                    double Tg = P / ng * tot.T_sum[(size_t)g * nb + k] / (m.C_tot * dx);
                    double qg = P / ng * tot.q_sum[(size_t)g * nb + k] / dx;
                    sT += Tg; sT2 += Tg * Tg; sq += qg; sq2 += qg * qg;
                }
                double Tm = 0, qm = 0;
                for (int g = 0; g < B; ++g) { Tm += tot.T_sum[(size_t)g * nb + k]; qm += tot.q_sum[(size_t)g * nb + k]; }
                Tm = P / Nd * Tm / (m.C_tot * dx);
                qm = P / Nd * qm / dx;
                if (T_mean) T_mean[k] = Tm;
                if (q_mean) q_mean[k] = qm;
                double vT = B > 1 ? (sT2 - sT * sT / B) / (B - 1.0) : 0.0;
                double vq = B > 1 ? (sq2 - sq * sq / B) / (B - 1.0) : 0.0;
                if (T_se) T_se[k] = sqrt(fmax(vT, 0.0) / B);
                if (q_se) q_se[k] = sqrt(fmax(vq, 0.0) / B);
            }
        }
        if (p->n_hj > 0) {
            for (int j = 0; j < p->n_hj; ++j) {
                double hm = tot.h_sum[j] / Nd;
                double hv = N > 1 ? (tot.h_sum2[j] - Nd * hm * hm) / (Nd - 1.0) : 0.0;
                if (h_mean) h_mean[j] = scale * hm;
                if (h_se) h_se[j] = scale * sqrt(fmax(hv, 0.0) / Nd);
            }
        }
        if (p->n_samples > 0 && grid_counts)
            memcpy(grid_counts, tot.grid, grid_cells(p) * sizeof(int64_t));
        /* steady maps: batch means over the n_batch groups; a cell's values
         * are per unit solid volume (solid area of the cell x thickness x
         * number of unit cells) */
        if (map_cells(p) > 0 && maps) {
            const int ny = p->map_ny, nz = p->map_nz, B = p->n_batch;
            const size_t cells = map_cells(p);
            const double dy = p->pitch / ny, dz = p->pitch / nz, c0 = 0.5 * p->pitch;
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j) {
                    const size_t i = (size_t)k * ny + j;
                    const double area = map_cell_solid(c0, p->radius, j * dy, (j + 1) * dy, k * dz, (k + 1) * dz);
                    const double V = area * p->L * p->cells_y * p->cells_z;
                    double sT = 0, sT2 = 0, sq = 0, sq2 = 0, Tt = 0, qt = 0;
                    for (int g = 0; g < B; ++g) {
                        /* particles 2q + e (e = 0, 1) below N with q = g mod B */
                        double ng = 0.0;
                        for (uint64_t e = 0; e < 2; ++e) {
                            uint64_t Q = N > e ? (N - e + 1) / 2 : 0;
                            ng += (double)(Q / B + ((uint64_t)g < Q % B ? 1 : 0));
                        }
                        if (ng <= 0) ng = 1;
                        double Tg = P / ng * tot.mT_sum[(size_t)g * cells + i] / (m.C_tot * V);
                        double qg = P / ng * tot.mq_sum[(size_t)g * cells + i] / V;
                        sT += Tg; sT2 += Tg * Tg; sq += qg; sq2 += qg * qg;
                        Tt += tot.mT_sum[(size_t)g * cells + i];
                        qt += tot.mq_sum[(size_t)g * cells + i];
                    }
                    double vT = B > 1 ? (sT2 - sT * sT / B) / (B - 1.0) : 0.0;
                    double vq = B > 1 ? (sq2 - sq * sq / B) / (B - 1.0) : 0.0;
                    /* a cell whose solid is below 1e-12 of its area counts as empty */
                    const int solid = area > 1e-12 * dy * dz;
                    maps[0 * cells + i] = solid ? P / Nd * Tt / (m.C_tot * V) : NAN;
                    maps[1 * cells + i] = solid ? sqrt(fmax(vT, 0.0) / B) : NAN;
                    maps[2 * cells + i] = solid ? P / Nd * qt / V : NAN;
                    maps[3 * cells + i] = solid ? sqrt(fmax(vq, 0.0) / B) : NAN;
                    maps[4 * cells + i] = solid ? area / (dy * dz) : 0.0;
                }
        }
    }
    for (int i = 0; i < nt; ++i) tally_free(&jobs[i].tally);
    tally_free(&tot);
    free(jobs);
    free(th);
    mat_free(&m);
    return rc;
}

/* Material tables as the oracle builds them (for host-side cross checks). */
int orc_material(const orc_problem* p, double* omega, double* v, double* tau, double* C, int cap)
{
    orc_mat m;
    memset(&m, 0, sizeof(m));
    if (mat_build(p, &m)) { mat_free(&m); return -1; }
    int n = m.n;
    if (omega && cap >= n) {
        memcpy(omega, m.omega, n * sizeof(double));
        memcpy(v, m.v, n * sizeof(double));
        memcpy(tau, m.tau, n * sizeof(double));
        memcpy(C, m.C, n * sizeof(double));
    }
    mat_free(&m);
    return n;
}

/* Inverse-CDF mode draw exposed for sampler tests: which = 0 emission, 1 scatter. */
int orc_draw_modes(const orc_problem* p, int which, const double* u, int n, int32_t* out)
{
    orc_mat m;
    memset(&m, 0, sizeof(m));
    if (mat_build(p, &m)) { mat_free(&m); return -1; }
    const double* cdf = which == 2 ? m.cdf_init : (which ? m.cdf_scat : m.cdf_emit);
    for (int i = 0; i < n; ++i) out[i] = draw_mode(cdf, m.n, u[i]);
    mat_free(&m);
    return 0;
}

/* First boundary along a ray, exposed for geometry tests. */
double orc_first_boundary(const orc_problem* p, const double pos[3], const double dir[3], int32_t* kind)
{
    orc_state s;
    memset(&s, 0, sizeof(s));
    s.x = pos[0]; s.y = pos[1]; s.z = pos[2];
    s.ox = dir[0]; s.oy = dir[1]; s.oz = dir[2];
    int k;
    double t = first_boundary(p, &s, &k);
    *kind = k;
    return t;
}

/* Initial states exposed for source tests: out[i*8 + ...] =
 * (sign, x, y, z, ox, oy, oz, t) plus modes[i]. */
int orc_emit(const orc_problem* p, uint64_t first, int n, double* out, int32_t* modes)
{
    orc_mat m;
    memset(&m, 0, sizeof(m));
    if (validate(p) || mat_build(p, &m)) { mat_free(&m); return -1; }
    for (int i = 0; i < n; ++i) {
        orc_state s;
        emit(p, &m, first + i, &s);
        double* o = out + (size_t)i * 8;
        o[0] = s.sign; o[1] = s.x;
        o[2] = s.cy * p->pitch + s.y; o[3] = s.cz * p->pitch + s.z;
        o[4] = s.ox; o[5] = s.oy; o[6] = s.oz; o[7] = s.t;
        if (modes) modes[i] = s.mode;
    }
    mat_free(&m);
    return 0;
}

/* The relaxation-event direction law for sampler tests: in = incoming
 * direction (unit), u_mu and u_phi the flight's third and fourth uniforms. */
void orc_scatter_direction(double g, const double in[3], double u_mu, double u_phi, double out[3])
{
    dir_axis(2, 2.0 * u_mu - 1.0, u_phi, &out[0], &out[1], &out[2]);
    if (g != 0.0) hg_direction(g, u_mu, u_phi, in[0], in[1], in[2], &out[0], &out[1], &out[2]);
}

int orc_sizeof_problem(void) { return (int)sizeof(orc_problem); }
int orc_sizeof_result(void) { return (int)sizeof(orc_result); }
int orc_sizeof_particle(void) { return (int)sizeof(orc_particle); }
