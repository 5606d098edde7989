/*
 * fdtd_oracle.c -- plain, slow, FP64 CPU oracle of the coupled Yee-FDTD +
 * two-term kinetic electron step of arXiv 2211.05647.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the entry-point smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA path: every coefficient below is rebuilt here from
 * the paper's formulas.
 *
 * What it computes, in the order of one time step n -> n+1:
 *   1. H^{n+1/2} from E^n with the Yee curl (Sec. 2, Eq. 1 and "in the same
 *      way" after Eq. 6) and the CPML auxiliaries psi_h (Eq. 7-12).
 *   2. delta f^{n+1/2} = alpha_j delta f^{n-1/2} + beta_j n E^n for every plasma
 *      cell: the Crank-Nicolson form of Eq. 22 printed in Sec. 5.2 (f_1x update).
 *   3. J^{n+1/2} = -e sum_j w_j delta f_j^{n+1/2}  (Eq. 24 and the Jx sum of Sec. 5.2).
 *   4. E^{n+1} with the Yee curl, psi_e and the -dt/eps0 J^{n+1/2} term (Eq. 2-6).
 *   5. a soft source g(t^{n+1}) added at the source node(s).
 *   6. first-order Mur ends (1-D only).
 * Threads: built plainly it is single-threaded.  Built with -fopenmp (the
 * all-core CPU baseline) the per-cell field loops and the per-slot kinetic
 * loop are shared among threads; every cell and slot is still computed by
 * the same expressions in the same order, so both builds give identical
 * results bit for bit.
 * Readings of the paper where it is garbled or silent (signs of the curl
 * coefficients, CPML kappa subscripts, psi time levels, the sign of e, the
 * velocity grids and the collision model) are the ones listed with the
 * design notes of this repository; each is restated next to the code that
 * uses it.
 *
 * Storage conventions (shared by nothing -- stated so a reader can check them):
 *   1-D: Ex on nodes k = 0..nz (nz+1 values), Hy on k+1/2, k = 0..nz-1.
 *   2-D TMz: Ez(i,j), Hx(i,j+1/2), Hy(i+1/2,j) all stored as nx*ny arrays at
 *            index j*nx+i.  Ez on i==0 or j==0 is a PEC node (held at 0); the
 *            nodes i==nx and j==ny are PEC ghosts (implicit 0, not stored).
 *   3-D: Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2),
 *        Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k) at index (k*ny+j)*nx+i, the same
 *        PEC convention on the low planes and ghosts on the high ones.
 * The kinetic current sits on the polarisation component: Ex (1-D, 3-D) or
 * Ez (2-D TMz).  Plasma cells are the polarisation nodes with density > 0,
 * except PEC / boundary nodes; they are numbered ("slots") in increasing
 * linear index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the step loops use (1 unless built with -fopenmp). */
int64_t or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* SI constants (CODATA 2018); e > 0 is the elementary charge magnitude. */
#define OR_C0 299792458.0
#define OR_QE 1.602176634e-19
#define OR_ME 9.1093837015e-31
#define OR_EPS0 8.8541878128e-12
#define OR_PI 3.14159265358979323846

/* Every field is 8 bytes so the ctypes mirror has no padding. */
typedef struct or_params {
    int64_t ndim;                 /* 1, 2 or 3 */
    int64_t nx, ny, nz;           /* cells per axis (1-D uses nz) */
    double dx;                    /* cell size on every axis (m) */
    double courant;               /* S, dt = S dx / c */
    int64_t cpml;                 /* CPML thickness in cells (2-D/3-D); 0 = none */
    double cpml_order, cpml_sigma_factor, cpml_kappa_max, cpml_alpha_min, cpml_alpha_max;
    int64_t mur;                  /* 1-D: first-order Mur at both ends, else PEC */
    int64_t src_kind;             /* 0 none, 1 Gaussian-modulated sine, 2 Gaussian */
    double src_amp, src_fc, src_tau, src_t0;
    int64_t src_i, src_j, src_k;  /* point-source node; 3-D sheet plane = src_k */
    int64_t src_sheet;            /* 3-D: 1 = sheet over [i0,i1) x [j0,j1) at k = src_k */
    int64_t sheet_i0, sheet_i1, sheet_j0, sheet_j1;
    int64_t vgrid;                /* 0 signed 1-D, 1 Cartesian (v_par, v_perp), 2 speed 3-D */
    int64_t nv, nv_perp;
    double te_ev, vmax_vth, nu0;
    int64_t nu_model;             /* 0: nu = N s |v| scaled to mean nu0; 1: nu = nu0; 2: s(v) from the table */
    int64_t nonlinear;            /* 1: add flux-form advection of delta f in v_par */
    int64_t f0_model;             /* 0: Maxwellian, 1: Druyvesteyn (same mean energy 3/2 e Te) */
    int64_t s_n;                  /* nu_model 2: points of the cross-section table */
    const double *s_speed;        /* ascending speeds (m/s) */
    const double *s_sigma;        /* s(v) at those speeds (any unit: only the shape matters) */
    int64_t evolve_f0;            /* speed grid: 1 = F0 evolves (heating + elastic collisions) */
    double mass_ratio;            /* m / M of the gas atom (elastic energy exchange) */
    double tg_ev;                 /* gas temperature (eV) */
} or_params;

typedef struct or_sim {
    or_params p;
    double dt;
    int64_t nx, ny, nz, ncell;    /* ncell = nodes of the 2-D/3-D arrays */
    double *f[6];                 /* Ex Ey Ez Hx Hy Hz (NULL where absent) */
    double *psi[12];              /* CPML auxiliaries, full-size, see psi_index() */
    double *pe_b[3], *pe_a[3], *pe_k[3];   /* per-axis CPML profile at E positions */
    double *ph_b[3], *ph_a[3], *ph_k[3];   /* ... at H positions */
    int64_t nslots, nnode;
    int64_t *slot_cell;
    double *dens;                 /* density per slot (m^-3) */
    double *df;                   /* delta f, [slot][node] */
    double *g0;                   /* evolve_f0: F0 - F0(table) per unit density, [slot][node] */
    double *jslot;                /* J^{n+1/2} per slot */
    double *jnode;                /* J on the polarisation array (0 off plasma) */
    double *v, *w, *f0, *f0p, *nu, *dV, *alpha, *beta;
    int64_t *mirror;              /* node with v_par -> -v_par */
    int64_t npar, nperp;
    double dvpar;
    int64_t step;
} or_sim;

enum { EX = 0, EY, EZ, HX, HY, HZ };

/* ---------------------------------------------------------------- source */

/* Soft source waveform.  Gaussian-modulated sine: the pulse of Table 3
 * (centre frequency f_c, time constant tau, shift t0); plain Gaussian: the
 * validation pulse shape of Eq. 14 (in time). */
double or_source(const or_params *p, double t)
{
    double u = (t - p->src_t0) / p->src_tau;
    if (p->src_kind == 1)
        return p->src_amp * sin(2.0 * OR_PI * p->src_fc * (t - p->src_t0)) * exp(-u * u);
    if (p->src_kind == 2)
        return p->src_amp * exp(-u * u);
    return 0.0;
}

/* ------------------------------------------------------- velocity tables */

/* Per-node tables of the kinetic update, for one velocity grid.
 *  v      : v_par of the node (the speed v for the speed grid)
 *  w      : quadrature weight of the current moment, J = -e sum_j w_j df_j
 *           (Eq. 24; speed grid: (4 pi / 3) v^3 gamma, the Jx sum of Sec. 5.2)
 *  f0     : normalised Maxwellian F0^ (integral over velocity space = 1)
 *  f0p    : dF0^/dv_par (speed grid: dF0^/dv) -- def_f_0 of Sec. 5.2
 *  nu     : elastic collision frequency, Eq. 23 nu = N s v with constant s
 *           scaled so that the grid's F0-weighted mean of nu is nu0, or nu0
 *  dV     : velocity-space volume element of the node
 *  alpha  : (2 - dt nu)/(2 + dt nu)                        (Sec. 5.2 update)
 *  beta   : 2 dt (e/m) f0p / (2 + dt nu)                     (Sec. 5.2 update)
 * Node order for the Cartesian grid: j = a * nv_perp + b, a the v_par index.
 * v_par nodes are midpoints of a uniform grid on [-vmax, vmax], written as
 * (a + 1/2 - nv/2) dv so that mirrored nodes are exact negatives. */
int64_t or_nnode_of(const or_params *p)
{
    if (p->vgrid == 1) return p->nv * p->nv_perp;
    return p->nv;
}

/* Druyvesteyn F0 of unit density: A exp(-(eps/eps0)^2), eps = m v^2 / 2.
 * Its mean energy is eps0 Gamma(5/4) / Gamma(3/4); it is set to (3/2) e Te so
 * that te_ev is the effective temperature, and A normalises the integral of
 * F0 over velocity space to 1. */
static double dr_eps0(double te_ev) { return 1.5 * OR_QE * te_ev * tgamma(0.75) / tgamma(1.25); }
static double dr_amp(double eps0) { return 1.0 / (OR_PI * tgamma(0.75) * pow(2.0 * eps0 / OR_ME, 1.5)); }
static double dr_f0(double A, double eps0, double v2)   /* F0 at |v|^2 = v2 */
{
    const double x = 0.5 * OR_ME * v2 / eps0;
    return A * exp(-x * x);
}

/* Cartesian 2-D grid, Druyvesteyn: the marginal over the third velocity
 * component t, h = int F0 dt, and its v_par derivative
 * dh/du = int F0'(r) u / r dt = -(2 m u / eps0^2) int eps F0 dt, by composite
 * Simpson on t in [0, 6 sqrt(2 eps0 / m)] (the integrand is even in t and
 * below 1e-300 of its peak beyond). */
static void dr_marginal2(double A, double eps0, double u, double w, double *h, double *dh)
{
    const int N = 20000;
    const double T = 6.0 * sqrt(2.0 * eps0 / OR_ME), dt = T / N;
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q <= N; ++q) {
        const double t = q * dt;
        const double v2 = u * u + w * w + t * t;
        const double f = dr_f0(A, eps0, v2);
        const double c = (q == 0 || q == N) ? 1.0 : (q % 2 ? 4.0 : 2.0);
        s0 += c * f;
        s1 += c * 0.5 * OR_ME * v2 * f;
    }
    *h = 2.0 * s0 * dt / 3.0;
    *dh = -(2.0 * OR_ME * u / (eps0 * eps0)) * 2.0 * s1 * dt / 3.0;
}

/* s(v) of the cross-section table, linear between points, constant beyond the ends */
static double table_sigma(const or_params *p, double v)
{
    const int64_t n = p->s_n;
    if (v <= p->s_speed[0]) return p->s_sigma[0];
    if (v >= p->s_speed[n - 1]) return p->s_sigma[n - 1];
    int64_t k = 0;
    while (p->s_speed[k + 1] < v) ++k;
    const double r = (v - p->s_speed[k]) / (p->s_speed[k + 1] - p->s_speed[k]);
    return p->s_sigma[k] + r * (p->s_sigma[k + 1] - p->s_sigma[k]);
}

/* Velocity-grid tables (Sec. 5.2, Eq. 20-24).  F0 enters through its value and
 * its v_par derivative on each grid: the 3-D F0 on the speed grid, its 1-D
 * marginal on the signed grid (Maxwellian: a Gaussian; Druyvesteyn:
 * (pi^{3/2}/2) A (2 eps0/m) erfc(m u^2 / (2 eps0)), derivative -2 pi u F0(|u|)),
 * its 2-D marginal on the Cartesian grid. */
void or_vtables(const or_params *p, double dt, double *v, double *w, double *f0,
                double *f0p, double *nu, double *dV, double *alpha, double *beta)
{
    const double vth = sqrt(OR_QE * p->te_ev / OR_ME);
    const double vmax = p->vmax_vth * vth;
    const int64_t nn = or_nnode_of(p);
    const int dru = p->f0_model == 1;
    const double eps0 = dr_eps0(p->te_ev), A = dr_amp(eps0);
    double *speed = (double *)malloc(sizeof(double) * nn);
    if (p->vgrid == 0) {
        const double dv = 2.0 * vmax / (double)p->nv;
        for (int64_t a = 0; a < p->nv; ++a) {
            double va = ((double)a + 0.5 - 0.5 * (double)p->nv) * dv;
            v[a] = va;
            if (dru) {
                f0[a] = 0.5 * pow(OR_PI, 1.5) * A * (2.0 * eps0 / OR_ME) * erfc(0.5 * OR_ME * va * va / eps0);
                f0p[a] = -2.0 * OR_PI * va * dr_f0(A, eps0, va * va);
            } else {
                double g = exp(-va * va / (2.0 * vth * vth)) / sqrt(2.0 * OR_PI * vth * vth);
                f0[a] = g;
                f0p[a] = -va / (vth * vth) * g;
            }
            w[a] = va * dv;
            dV[a] = dv;
            speed[a] = fabs(va);
        }
    } else if (p->vgrid == 1) {
        const double dvp = 2.0 * vmax / (double)p->nv;
        const double dvq = 2.0 * vmax / (double)p->nv_perp;
        for (int64_t a = 0; a < p->nv; ++a) {
            double va = ((double)a + 0.5 - 0.5 * (double)p->nv) * dvp;
            for (int64_t b = 0; b < p->nv_perp; ++b) {
                double vb = ((double)b + 0.5 - 0.5 * (double)p->nv_perp) * dvq;
                int64_t j = a * p->nv_perp + b;
                v[j] = va;
                if (dru) {
                    dr_marginal2(A, eps0, va, vb, &f0[j], &f0p[j]);
                } else {
                    double g = exp(-(va * va + vb * vb) / (2.0 * vth * vth)) / (2.0 * OR_PI * vth * vth);
                    f0[j] = g;
                    f0p[j] = -va / (vth * vth) * g;
                }
                w[j] = va * dvp * dvq;
                dV[j] = dvp * dvq;
                speed[j] = sqrt(va * va + vb * vb);
            }
        }
    } else {
        const double gam = vmax / (double)p->nv;
        for (int64_t k = 0; k < p->nv; ++k) {
            double vk = ((double)k + 0.5) * gam;
            v[k] = vk;
            if (dru) {
                const double g = dr_f0(A, eps0, vk * vk);
                f0[k] = g;
                f0p[k] = -(OR_ME * OR_ME * vk * vk * vk / (eps0 * eps0)) * g;   /* dF0/dv */
            } else {
                double g = exp(-vk * vk / (2.0 * vth * vth)) / pow(2.0 * OR_PI * vth * vth, 1.5);
                f0[k] = g;
                f0p[k] = -vk / (vth * vth) * g;
            }
            w[k] = (4.0 * OR_PI / 3.0) * vk * vk * vk * gam;
            dV[k] = 4.0 * OR_PI * vk * vk * gam;
            speed[k] = vk;
        }
    }
    /* collision frequency (Eq. 23): nu = N s(v) |v|; N fixed by the F0-weighted
     * mean of nu = nu0; s constant (model 0) or tabulated (model 2) */
    double num = 0.0, den = 0.0;
    for (int64_t j = 0; j < nn; ++j) {
        const double sv = (p->nu_model == 2 ? table_sigma(p, speed[j]) : 1.0) * speed[j];
        num += sv * f0[j] * dV[j];
        den += f0[j] * dV[j];
    }
    const double mean_sv = num / den;
    for (int64_t j = 0; j < nn; ++j) {
        const double sv = (p->nu_model == 2 ? table_sigma(p, speed[j]) : 1.0) * speed[j];
        nu[j] = (p->nu_model == 1) ? p->nu0 : p->nu0 * sv / mean_sv;
        alpha[j] = (2.0 - dt * nu[j]) / (2.0 + dt * nu[j]);
        beta[j] = 2.0 * dt * (OR_QE / OR_ME) * f0p[j] / (2.0 + dt * nu[j]);
    }
    free(speed);
}

/* --------------------------------------------------------- CPML profiles */

/* One axis of n cells with an L-cell CPML on each end, at E positions
 * (x = i dx) or H positions (x = (i + 1/2) dx), i = 0..n-1.
 * rho = depth into the layer from its inner interface (Eq. 12 notation);
 * sigma = sigma_max (rho/delta)^order, kappa = 1 + (kappa_max-1)(rho/delta)^order,
 * alpha = alpha_min + (alpha_max-alpha_min)(1 - rho/delta)        (Eq. 12),
 * sigma_max = sigma_factor (order+1) / (150 pi dx)                 (Eq. 11),
 * b = exp(-(sigma/kappa + alpha) dt/eps0)                          (Eq. 9),
 * a = sigma (b-1) / (dx (sigma kappa + alpha kappa^2))             (Eq. 10).
 * Outside the layers kappa = 1 and a = b = 0 (psi stays 0 there).
 * The magnetic profiles use the same expressions: with sigma_m = mu0/eps0 sigma
 * and alpha_m = mu0/eps0 alpha the ratio mu0/eps0 cancels in a and b. */
void or_cpml_profile(const or_params *p, double dt, int64_t n, int at_h,
                     double *b, double *a, double *kap)
{
    const int64_t L = p->cpml;
    const double dx = p->dx;
    const double delta = (double)L * dx;
    const double smax = p->cpml_sigma_factor * (p->cpml_order + 1.0) / (150.0 * OR_PI * dx);
    for (int64_t i = 0; i < n; ++i) {
        double x = ((double)i + (at_h ? 0.5 : 0.0)) * dx;
        double rho = 0.0;
        int in = 0;
        if (L > 0 && x < delta) { rho = delta - x; in = 1; }
        if (L > 0 && x > (double)(n - L) * dx) { rho = x - (double)(n - L) * dx; in = 1; }
        if (!in) { b[i] = 0.0; a[i] = 0.0; kap[i] = 1.0; continue; }
        double r = rho / delta;
        double rn = pow(r, p->cpml_order);
        double sig = smax * rn;
        double k = 1.0 + (p->cpml_kappa_max - 1.0) * rn;
        double al = p->cpml_alpha_min + (p->cpml_alpha_max - p->cpml_alpha_min) * (1.0 - r);
        double bb = exp(-(sig / k + al) * dt / OR_EPS0);
        double den = dx * (sig * k + al * k * k);
        b[i] = bb;
        a[i] = (sig > 0.0 && den > 0.0) ? sig * (bb - 1.0) / den : 0.0;
        kap[i] = k;
    }
}

/* --------------------------------------------------------------- helpers */

static int64_t pol_component(const or_params *p) { return p->ndim == 2 ? EZ : EX; }

static int64_t pol_len(const or_sim *s) { return s->p.ndim == 1 ? s->nz + 1 : s->ncell; }

/* Is polarisation node c a node whose E is updated by the curl (so it may
 * carry plasma)?  1-D: 1..nz-1.  2-D Ez: i>=1, j>=1.  3-D Ex: j>=1, k>=1. */
static int pol_updated(const or_sim *s, int64_t c)
{
    if (s->p.ndim == 1) return c >= 1 && c <= s->nz - 1;
    int64_t i = c % s->nx, j = (c / s->nx) % s->ny, k = c / (s->nx * s->ny);
    if (s->p.ndim == 2) return i >= 1 && j >= 1;
    (void)i;
    return j >= 1 && k >= 1;
}

int64_t or_field_len(const or_sim *s, int which)
{
    if (which < 0 || which > 5) return 0;
    return s->f[which] ? (s->p.ndim == 1 ? (which == EX ? s->nz + 1 : s->nz) : s->ncell) : 0;
}

/* ---------------------------------------------------------------- create */

or_sim *or_create(const or_params *p, const double *density)
{
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->p = *p;
    s->dt = p->courant * p->dx / OR_C0;
    s->nx = p->ndim >= 2 ? p->nx : 1;
    s->ny = p->ndim >= 2 ? p->ny : 1;
    s->nz = p->ndim == 2 ? 1 : p->nz;
    if (p->ndim == 1) {
        s->ncell = s->nz + 1;
        s->f[EX] = (double *)calloc((size_t)(s->nz + 1), sizeof(double));
        s->f[HY] = (double *)calloc((size_t)s->nz, sizeof(double));
    } else {
        s->ncell = s->nx * s->ny * s->nz;
        int comps2[3] = {EZ, HX, HY};
        if (p->ndim == 2) {
            for (int c = 0; c < 3; ++c) s->f[comps2[c]] = (double *)calloc((size_t)s->ncell, sizeof(double));
        } else {
            for (int c = 0; c < 6; ++c) s->f[c] = (double *)calloc((size_t)s->ncell, sizeof(double));
        }
        if (p->cpml > 0) {
            int npsi = p->ndim == 2 ? 4 : 12;
            /* calloc'd pages that are never written (outside the layers) are
             * never touched: psi is only updated where the profile is nonzero. */
            for (int q = 0; q < npsi; ++q) s->psi[q] = (double *)calloc((size_t)s->ncell, sizeof(double));
            int64_t n[3] = {s->nx, s->ny, s->nz};
            for (int ax = 0; ax < p->ndim; ++ax) {
                s->pe_b[ax] = (double *)malloc(sizeof(double) * n[ax]);
                s->pe_a[ax] = (double *)malloc(sizeof(double) * n[ax]);
                s->pe_k[ax] = (double *)malloc(sizeof(double) * n[ax]);
                s->ph_b[ax] = (double *)malloc(sizeof(double) * n[ax]);
                s->ph_a[ax] = (double *)malloc(sizeof(double) * n[ax]);
                s->ph_k[ax] = (double *)malloc(sizeof(double) * n[ax]);
                or_cpml_profile(p, s->dt, n[ax], 0, s->pe_b[ax], s->pe_a[ax], s->pe_k[ax]);
                or_cpml_profile(p, s->dt, n[ax], 1, s->ph_b[ax], s->ph_a[ax], s->ph_k[ax]);
            }
        }
    }
    /* plasma cells */
    s->nnode = or_nnode_of(p);
    int64_t np = pol_len(s);
    s->jnode = (double *)calloc((size_t)np, sizeof(double));
    s->nslots = 0;
    if (density) {
        for (int64_t c = 0; c < np; ++c)
            if (density[c] > 0.0 && pol_updated(s, c)) s->nslots++;
    }
    s->slot_cell = (int64_t *)malloc(sizeof(int64_t) * (s->nslots ? s->nslots : 1));
    s->dens = (double *)malloc(sizeof(double) * (s->nslots ? s->nslots : 1));
    s->jslot = (double *)calloc((size_t)(s->nslots ? s->nslots : 1), sizeof(double));
    s->df = (double *)calloc((size_t)((s->nslots ? s->nslots : 1) * s->nnode), sizeof(double));
    s->g0 = (double *)calloc((size_t)((s->nslots ? s->nslots : 1) * s->nnode), sizeof(double));
    int64_t q = 0;
    if (density) {
        for (int64_t c = 0; c < np; ++c)
            if (density[c] > 0.0 && pol_updated(s, c)) {
                s->slot_cell[q] = c;
                s->dens[q] = density[c];
                ++q;
            }
    }
    int64_t nn = s->nnode;
    s->v = malloc(sizeof(double) * nn); s->w = malloc(sizeof(double) * nn);
    s->f0 = malloc(sizeof(double) * nn); s->f0p = malloc(sizeof(double) * nn);
    s->nu = malloc(sizeof(double) * nn); s->dV = malloc(sizeof(double) * nn);
    s->alpha = malloc(sizeof(double) * nn); s->beta = malloc(sizeof(double) * nn);
    s->mirror = malloc(sizeof(int64_t) * nn);
    or_vtables(p, s->dt, s->v, s->w, s->f0, s->f0p, s->nu, s->dV, s->alpha, s->beta);
    s->npar = p->nv;
    s->nperp = p->vgrid == 1 ? p->nv_perp : 1;
    {
        const double vth = sqrt(OR_QE * p->te_ev / OR_ME);
        s->dvpar = 2.0 * p->vmax_vth * vth / (double)p->nv;
    }
    for (int64_t a = 0; a < s->npar; ++a)
        for (int64_t b = 0; b < s->nperp; ++b)
            s->mirror[a * s->nperp + b] = (s->npar - 1 - a) * s->nperp + b;
    return s;
}

void or_destroy(or_sim *s)
{
    if (!s) return;
    for (int c = 0; c < 6; ++c) free(s->f[c]);
    for (int q = 0; q < 12; ++q) free(s->psi[q]);
    for (int ax = 0; ax < 3; ++ax) {
        free(s->pe_b[ax]); free(s->pe_a[ax]); free(s->pe_k[ax]);
        free(s->ph_b[ax]); free(s->ph_a[ax]); free(s->ph_k[ax]);
    }
    free(s->slot_cell); free(s->dens); free(s->jslot); free(s->df); free(s->g0); free(s->jnode);
    free(s->v); free(s->w); free(s->f0); free(s->f0p); free(s->nu); free(s->dV);
    free(s->alpha); free(s->beta); free(s->mirror);
    free(s);
}

double or_dt(const or_sim *s) { return s->dt; }
int64_t or_nslots(const or_sim *s) { return s->nslots; }
int64_t or_nnode(const or_sim *s) { return s->nnode; }
int64_t or_steps_done(const or_sim *s) { return s->step; }
void or_slot_cells(const or_sim *s, int64_t *out) { memcpy(out, s->slot_cell, sizeof(int64_t) * s->nslots); }

/* which: 0..5 fields, 6 = J per slot, 7 = delta f [slot][node], 8 = F0 correction [slot][node] */
int or_get(const or_sim *s, int which, double *out)
{
    if (which >= 0 && which <= 5) {
        int64_t n = or_field_len(s, which);
        if (!n) return -1;
        memcpy(out, s->f[which], sizeof(double) * n);
        return 0;
    }
    if (which == 6) { memcpy(out, s->jslot, sizeof(double) * s->nslots); return 0; }
    if (which == 7) { memcpy(out, s->df, sizeof(double) * s->nslots * s->nnode); return 0; }
    if (which == 8) { memcpy(out, s->g0, sizeof(double) * s->nslots * s->nnode); return 0; }
    return -1;
}

int or_set(or_sim *s, int which, const double *in)
{
    if (which >= 0 && which <= 5) {
        int64_t n = or_field_len(s, which);
        if (!n) return -1;
        memcpy(s->f[which], in, sizeof(double) * n);
        return 0;
    }
    if (which == 6) {
        memcpy(s->jslot, in, sizeof(double) * s->nslots);
        for (int64_t q = 0; q < s->nslots; ++q) s->jnode[s->slot_cell[q]] = s->jslot[q];
        return 0;
    }
    if (which == 7) { memcpy(s->df, in, sizeof(double) * s->nslots * s->nnode); return 0; }
    if (which == 8) { memcpy(s->g0, in, sizeof(double) * s->nslots * s->nnode); return 0; }
    return -1;
}

/* --------------------------------------------------------- kinetic step */

/* Sec. 5.2 update of the anisotropic part for every plasma cell, using E^n:
 *   (2 + dt nu_j) df_j^{n+1/2} = (2 - dt nu_j) df_j^{n-1/2} + 2 dt (e/m) F0'_j n E^n
 * i.e. Crank-Nicolson on Eq. 22 with e > 0 the charge magnitude (electrons feel
 * -eE), then J^{n+1/2} = -e sum_j w_j df_j^{n+1/2} (Eq. 24).
 * Nonlinear mode (v_par grids only): the advection of delta f itself by the
 * acceleration a = -(e/m) E is added in flux form with donor-cell fluxes and
 * zero flux through +-vmax, which conserves sum_j df_j dV_j exactly; elastic
 * collisions then relax only the part of delta f that is odd in v_par:
 *   odd^{n+1/2}  = alpha odd^{n-1/2} + beta n E + 2 dt A_odd / (2 + dt nu)
 *   even^{n+1/2} = even^{n-1/2} + dt A_even
 * with A_j = -(Phi_{a+1/2} - Phi_{a-1/2}) / dv_par.  (The linear mode is the
 * paper's model; with delta f odd it is the same update without A.) */
/* Isotropic F0 evolution on the speed grid (the F0 equation of the two-term
 * expansion, Sec. 5.2, without the spatial term of the local model):
 *   dF0/dt = (e E / (3 m v^2)) d/dv (v^2 F1) + C0(F0),
 *   C0 = (m/M) (1/v^2) d/dv [ v^3 nu (F0 + (k Tg / (m v)) dF0/dv) ]  (elastic).
 * F0 = F0(table) + g with g per unit density; F1 = delta f / n.  One step,
 * with E = E^n, F1 and g at n - 1/2 on entry:
 *  1. F0' = F0'(table) + central differences of g (g mirrored at v = 0,
 *     zero beyond the last node);
 *  2. delta f^{n+1/2} = alpha delta f^{n-1/2} + 2 dt (e/m) F0' / (2 + dt nu) n E;
 *  3. J from the new delta f;
 *  4. g += dt (heating + collisions), both in flux form over the cell edges
 *     v_{k+1/2} = (k+1) gamma with zero flux through v = 0 and v_max: heating
 *     flux (v_k^3 F1_k + v_{k+1}^3 F1_{k+1}) / (2 v_{k+1/2}) of the time-centred
 *     F1 = (delta f^{n-1/2} + delta f^{n+1/2}) / (2 n); collision flux
 *     (m/M) v^3 nu (F0 + (k Tg/(m v)) dF0/dv) at the edge with edge averages of
 *     F0 and nu and the one-cell difference of F0, from the F0 at n - 1/2.
 * Rows are plain arrays of nn nodes; fold, old, hflux, cflux are scratch. */
static void evolve_row(const or_params *p, double dt, const double *v, const double *f0, const double *f0p,
                       const double *nu, const double *alpha, const double *w, double n, double E, double *row,
                       double *g, double *old, double *hflux, double *cflux, double *J)
{
    const int64_t nn = p->nv;
    const double gam = v[0] * 2.0;     /* nodes at (k + 1/2) gamma */
    const double qm = OR_QE / OR_ME;
    memcpy(old, row, sizeof(double) * nn);
    for (int64_t k = 0; k < nn; ++k) {
        const double gl = k > 0 ? g[k - 1] : g[0];
        const double gr = k + 1 < nn ? g[k + 1] : 0.0;
        const double d = f0p[k] + (gr - gl) / (2.0 * gam);
        row[k] = alpha[k] * row[k] + 2.0 * dt * qm * d / (2.0 + dt * nu[k]) * n * E;
    }
    double j = 0.0;
    for (int64_t k = 0; k < nn; ++k) j += w[k] * row[k];
    *J = -OR_QE * j;
    const double kTg_m = OR_QE * p->tg_ev / OR_ME;
    for (int64_t k = 0; k + 1 < nn; ++k) {    /* edge k + 1/2 */
        const double ve = (double)(k + 1) * gam;
        const double a0 = v[k] * v[k] * v[k] * 0.5 * (old[k] + row[k]) / n;
        const double a1 = v[k + 1] * v[k + 1] * v[k + 1] * 0.5 * (old[k + 1] + row[k + 1]) / n;
        hflux[k] = 0.5 * (a0 + a1) / ve;
        const double F0k = f0[k] + g[k], F0k1 = f0[k + 1] + g[k + 1];
        const double nue = 0.5 * (nu[k] + nu[k + 1]);
        cflux[k] = p->mass_ratio * ve * ve * ve * nue * (0.5 * (F0k + F0k1) + kTg_m / ve * (F0k1 - F0k) / gam);
    }
    for (int64_t k = 0; k < nn; ++k) {
        const double hr = k + 1 < nn ? hflux[k] : 0.0, hl = k > 0 ? hflux[k - 1] : 0.0;
        const double cr = k + 1 < nn ? cflux[k] : 0.0, cl = k > 0 ? cflux[k - 1] : 0.0;
        const double v2g = v[k] * v[k] * gam;
        g[k] += dt * ((qm * E / 3.0) * (hr - hl) / v2g + (cr - cl) / v2g);
    }
}

static void kinetic_step(or_sim *s)
{
    const int64_t nn = s->nnode;
    double *Ep = s->f[pol_component(&s->p)];
    const double dt = s->dt;
#pragma omp parallel
    {
    double *old = (double *)malloc(sizeof(double) * nn);   /* scratch rows, one pair per thread */
    double *A = (double *)malloc(sizeof(double) * nn);
#pragma omp for schedule(static)
    for (int64_t q = 0; q < s->nslots; ++q) {
        const int64_t c = s->slot_cell[q];
        const double E = Ep[c];
        const double nE = s->dens[q] * E;
        double *row = s->df + q * nn;
        if (s->p.evolve_f0) {
            double *scratch = (double *)malloc(sizeof(double) * 2 * nn);
            double J;
            evolve_row(&s->p, dt, s->v, s->f0, s->f0p, s->nu, s->alpha, s->w, s->dens[q], E, row, s->g0 + q * nn,
                       old, scratch, scratch + nn, &J);
            free(scratch);
            s->jslot[q] = J;
            s->jnode[c] = J;
            continue;
        }
        if (!s->p.nonlinear) {
            for (int64_t j = 0; j < nn; ++j) row[j] = s->alpha[j] * row[j] + s->beta[j] * nE;
        } else {
            const double acc = -(OR_QE / OR_ME) * E;
            memcpy(old, row, sizeof(double) * nn);
            for (int64_t a = 0; a < s->npar; ++a)
                for (int64_t b = 0; b < s->nperp; ++b) {
                    /* donor-cell flux through the faces a-1/2 and a+1/2 */
                    double fl_lo = 0.0, fl_hi = 0.0;
                    if (a > 0) {
                        double up = acc > 0.0 ? old[(a - 1) * s->nperp + b] : old[a * s->nperp + b];
                        fl_lo = acc * up;
                    }
                    if (a < s->npar - 1) {
                        double up = acc > 0.0 ? old[a * s->nperp + b] : old[(a + 1) * s->nperp + b];
                        fl_hi = acc * up;
                    }
                    A[a * s->nperp + b] = -(fl_hi - fl_lo) / s->dvpar;
                }
            for (int64_t j = 0; j < nn; ++j) {
                int64_t m = s->mirror[j];
                double odd = 0.5 * (old[j] - old[m]), even = 0.5 * (old[j] + old[m]);
                double aodd = 0.5 * (A[j] - A[m]), aeven = 0.5 * (A[j] + A[m]);
                row[j] = even + dt * aeven + s->alpha[j] * odd + s->beta[j] * nE +
                         2.0 * dt * aodd / (2.0 + dt * s->nu[j]);
            }
        }
        double J = 0.0;
        for (int64_t j = 0; j < nn; ++j) J += s->w[j] * row[j];
        J *= -OR_QE;
        s->jslot[q] = J;
        s->jnode[c] = J;
    }
    free(old);
    free(A);
    }
}

/* ---------------------------------------------------------- field steps */

#define ID2(i, j) ((j) * nx + (i))
#define ID3(i, j, k) (((k) * ny + (j)) * nx + (i))

static void step1d(or_sim *s)
{
    const int64_t nz = s->nz;
    double *ex = s->f[EX], *hy = s->f[HY];
    const double dt = s->dt, dz = s->p.dx;
    const double mu0 = 1.0 / (OR_EPS0 * OR_C0 * OR_C0);
    /* H: mu0 dHy/dt = -(curl E)_y = -dEx/dz */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k) hy[k] -= dt / (mu0 * dz) * (ex[k + 1] - ex[k]);
    const double e0 = ex[0], e1 = ex[1], en = ex[nz], enm1 = ex[nz - 1];
    kinetic_step(s);
    /* E: eps0 dEx/dt = (curl H)_x - Jx = -dHy/dz - Jx  (Eq. 1, 2, 6) */
#pragma omp parallel for schedule(static)
    for (int64_t k = 1; k < nz; ++k)
        ex[k] += -dt / (OR_EPS0 * dz) * (hy[k] - hy[k - 1]) - dt / OR_EPS0 * s->jnode[k];
    if (s->p.src_kind) ex[s->p.src_k] += or_source(&s->p, (double)(s->step + 1) * dt);
    if (s->p.mur) {
        /* first-order Mur: E0^{n+1} = E1^n + m (E1^{n+1} - E0^n) */
        const double m = (OR_C0 * dt - dz) / (OR_C0 * dt + dz);
        ex[0] = e1 + m * (ex[1] - e0);
        ex[nz] = enm1 + m * (ex[nz - 1] - en);
    }
}

static void step2d(or_sim *s)
{
    const int64_t nx = s->nx, ny = s->ny;
    double *ez = s->f[EZ], *hx = s->f[HX], *hy = s->f[HY];
    const double dt = s->dt, dx = s->p.dx;
    const double mu0 = 1.0 / (OR_EPS0 * OR_C0 * OR_C0);
    const int pml = s->p.cpml > 0;
    /* psi slots for 2-D: 0 psi_ez_x, 1 psi_ez_y, 2 psi_hx_y, 3 psi_hy_x */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            double e = ez[ID2(i, j)];
            double dEy = (j + 1 < ny ? ez[ID2(i, j + 1)] : 0.0) - e;   /* dEz/dy at (i, j+1/2) */
            double dEx = (i + 1 < nx ? ez[ID2(i + 1, j)] : 0.0) - e;   /* dEz/dx at (i+1/2, j) */
            /* mu0 dHx/dt = -dEz/dy ; mu0 dHy/dt = +dEz/dx */
            if (pml) {
                double *py = &s->psi[2][ID2(i, j)], *px = &s->psi[3][ID2(i, j)];
                if (s->ph_b[1][j] != 0.0 || s->ph_a[1][j] != 0.0) *py = s->ph_b[1][j] * *py + s->ph_a[1][j] * dEy;
                if (s->ph_b[0][i] != 0.0 || s->ph_a[0][i] != 0.0) *px = s->ph_b[0][i] * *px + s->ph_a[0][i] * dEx;
                hx[ID2(i, j)] -= dt / (mu0 * dx) * dEy / s->ph_k[1][j] + dt / mu0 * *py;
                hy[ID2(i, j)] += dt / (mu0 * dx) * dEx / s->ph_k[0][i] + dt / mu0 * *px;
            } else {
                hx[ID2(i, j)] -= dt / (mu0 * dx) * dEy;
                hy[ID2(i, j)] += dt / (mu0 * dx) * dEx;
            }
        }
    kinetic_step(s);
    /* eps0 dEz/dt = dHy/dx - dHx/dy - Jz */
#pragma omp parallel for schedule(static)
    for (int64_t j = 1; j < ny; ++j)
        for (int64_t i = 1; i < nx; ++i) {
            double dHx = hy[ID2(i, j)] - hy[ID2(i - 1, j)];
            double dHy = hx[ID2(i, j)] - hx[ID2(i, j - 1)];
            double upd;
            if (pml) {
                double *px = &s->psi[0][ID2(i, j)], *py = &s->psi[1][ID2(i, j)];
                if (s->pe_b[0][i] != 0.0 || s->pe_a[0][i] != 0.0) *px = s->pe_b[0][i] * *px + s->pe_a[0][i] * dHx;
                if (s->pe_b[1][j] != 0.0 || s->pe_a[1][j] != 0.0) *py = s->pe_b[1][j] * *py + s->pe_a[1][j] * dHy;
                upd = dt / (OR_EPS0 * dx) * (dHx / s->pe_k[0][i] - dHy / s->pe_k[1][j]) + dt / OR_EPS0 * (*px - *py);
            } else {
                upd = dt / (OR_EPS0 * dx) * (dHx - dHy);
            }
            ez[ID2(i, j)] += upd - dt / OR_EPS0 * s->jnode[ID2(i, j)];
        }
    if (s->p.src_kind) ez[ID2(s->p.src_i, s->p.src_j)] += or_source(&s->p, (double)(s->step + 1) * dt);
}

/* psi index for 3-D: field f (0..5) and derivative axis a: the two axes of
 * the curl of component f are the other two; slot = 2*f + (a == first other ? 0 : 1). */
static int psi3(int f, int a)
{
    int c = f % 3;                 /* x, y, z of the component */
    int o1 = (c + 1) % 3, o2 = (c + 2) % 3;
    int lo = o1 < o2 ? o1 : o2;
    return 2 * f + (a == lo ? 0 : 1);
}

static inline double psi_upd(double *psi, double b, double a, double d)
{
    if (b != 0.0 || a != 0.0) *psi = b * *psi + a * d;
    return *psi;
}

static void step3d(or_sim *s)
{
    const int64_t nx = s->nx, ny = s->ny, nz = s->nz;
    double *ex = s->f[EX], *ey = s->f[EY], *ez = s->f[EZ];
    double *hx = s->f[HX], *hy = s->f[HY], *hz = s->f[HZ];
    const double dt = s->dt, dx = s->p.dx;
    const double mu0 = 1.0 / (OR_EPS0 * OR_C0 * OR_C0);
    const double ch = dt / (mu0 * dx), cph = dt / mu0;
    const double ce = dt / (OR_EPS0 * dx), cpe = dt / OR_EPS0;
    const int pml = s->p.cpml > 0;
#define EV(arr, i, j, k) (((i) < nx && (j) < ny && (k) < nz) ? arr[ID3(i, j, k)] : 0.0)
    /* H update:  mu0 dH/dt = -curl E */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t c = ID3(i, j, k);
                double dEz_y = EV(ez, i, j + 1, k) - ez[c];
                double dEy_z = EV(ey, i, j, k + 1) - ey[c];
                double dEx_z = EV(ex, i, j, k + 1) - ex[c];
                double dEz_x = EV(ez, i + 1, j, k) - ez[c];
                double dEy_x = EV(ey, i + 1, j, k) - ey[c];
                double dEx_y = EV(ex, i, j + 1, k) - ex[c];
                if (pml) {
                    double pxy = psi_upd(&s->psi[psi3(HX, 1)][c], s->ph_b[1][j], s->ph_a[1][j], dEz_y);
                    double pxz = psi_upd(&s->psi[psi3(HX, 2)][c], s->ph_b[2][k], s->ph_a[2][k], dEy_z);
                    double pyz = psi_upd(&s->psi[psi3(HY, 2)][c], s->ph_b[2][k], s->ph_a[2][k], dEx_z);
                    double pyx = psi_upd(&s->psi[psi3(HY, 0)][c], s->ph_b[0][i], s->ph_a[0][i], dEz_x);
                    double pzx = psi_upd(&s->psi[psi3(HZ, 0)][c], s->ph_b[0][i], s->ph_a[0][i], dEy_x);
                    double pzy = psi_upd(&s->psi[psi3(HZ, 1)][c], s->ph_b[1][j], s->ph_a[1][j], dEx_y);
                    hx[c] -= ch * (dEz_y / s->ph_k[1][j] - dEy_z / s->ph_k[2][k]) + cph * (pxy - pxz);
                    hy[c] -= ch * (dEx_z / s->ph_k[2][k] - dEz_x / s->ph_k[0][i]) + cph * (pyz - pyx);
                    hz[c] -= ch * (dEy_x / s->ph_k[0][i] - dEx_y / s->ph_k[1][j]) + cph * (pzx - pzy);
                } else {
                    hx[c] -= ch * (dEz_y - dEy_z);
                    hy[c] -= ch * (dEx_z - dEz_x);
                    hz[c] -= ch * (dEy_x - dEx_y);
                }
            }
    kinetic_step(s);
    /* E update:  eps0 dE/dt = curl H - J  (J on Ex only) */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t c = ID3(i, j, k);
                double dHz_y = j > 0 ? hz[c] - hz[ID3(i, j - 1, k)] : 0.0;
                double dHy_z = k > 0 ? hy[c] - hy[ID3(i, j, k - 1)] : 0.0;
                double dHx_z = k > 0 ? hx[c] - hx[ID3(i, j, k - 1)] : 0.0;
                double dHz_x = i > 0 ? hz[c] - hz[ID3(i - 1, j, k)] : 0.0;
                double dHy_x = i > 0 ? hy[c] - hy[ID3(i - 1, j, k)] : 0.0;
                double dHx_y = j > 0 ? hx[c] - hx[ID3(i, j - 1, k)] : 0.0;
                if (pml) {
                    if (j > 0 && k > 0) {
                        double pxy = psi_upd(&s->psi[psi3(EX, 1)][c], s->pe_b[1][j], s->pe_a[1][j], dHz_y);
                        double pxz = psi_upd(&s->psi[psi3(EX, 2)][c], s->pe_b[2][k], s->pe_a[2][k], dHy_z);
                        ex[c] += ce * (dHz_y / s->pe_k[1][j] - dHy_z / s->pe_k[2][k]) + cpe * (pxy - pxz) -
                                 cpe * s->jnode[c];
                    }
                    if (i > 0 && k > 0) {
                        double pyz = psi_upd(&s->psi[psi3(EY, 2)][c], s->pe_b[2][k], s->pe_a[2][k], dHx_z);
                        double pyx = psi_upd(&s->psi[psi3(EY, 0)][c], s->pe_b[0][i], s->pe_a[0][i], dHz_x);
                        ey[c] += ce * (dHx_z / s->pe_k[2][k] - dHz_x / s->pe_k[0][i]) + cpe * (pyz - pyx);
                    }
                    if (i > 0 && j > 0) {
                        double pzx = psi_upd(&s->psi[psi3(EZ, 0)][c], s->pe_b[0][i], s->pe_a[0][i], dHy_x);
                        double pzy = psi_upd(&s->psi[psi3(EZ, 1)][c], s->pe_b[1][j], s->pe_a[1][j], dHx_y);
                        ez[c] += ce * (dHy_x / s->pe_k[0][i] - dHx_y / s->pe_k[1][j]) + cpe * (pzx - pzy);
                    }
                } else {
                    if (j > 0 && k > 0) ex[c] += ce * (dHz_y - dHy_z) - cpe * s->jnode[c];
                    if (i > 0 && k > 0) ey[c] += ce * (dHx_z - dHz_x);
                    if (i > 0 && j > 0) ez[c] += ce * (dHy_x - dHx_y);
                }
            }
    if (s->p.src_kind) {
        double g = or_source(&s->p, (double)(s->step + 1) * dt);
        if (s->p.src_sheet) {
            for (int64_t j = s->p.sheet_j0; j < s->p.sheet_j1; ++j)
                for (int64_t i = s->p.sheet_i0; i < s->p.sheet_i1; ++i) ex[ID3(i, j, s->p.src_k)] += g;
        } else {
            ex[ID3(s->p.src_i, s->p.src_j, s->p.src_k)] += g;
        }
    }
#undef EV
}

void or_step(or_sim *s, int64_t n)
{
    for (int64_t t = 0; t < n; ++t) {
        if (s->p.ndim == 1) step1d(s);
        else if (s->p.ndim == 2) step2d(s);
        else step3d(s);
        s->step++;
    }
}

/* ------------------------------------------------------- diagnostics */

/* out[0] discrete EM energy W = sum eps0/2 E^2 dV + mu0/2 H . H_next dV, where
 *        H_next is H advanced once more by the vacuum curl of the current E
 *        (without CPML terms).  In a lossless PEC cavity W is invariant.
 * out[1] particle-number perturbation sum_slots sum_j df_j dV_j
 * out[2] max over plasma cells of |sum_j df_j dV_j|
 * out[3] sum_slots sum_j |df_j| dV_j
 * out[4] 1 if every field, psi and df value is finite, else 0
 * out[5] plain energy sum eps0/2 E^2 dV + mu0/2 H^2 dV */
void or_diag(const or_sim *s, double *out)
{
    const double dt = s->dt, dx = s->p.dx;
    const double mu0 = 1.0 / (OR_EPS0 * OR_C0 * OR_C0);
    const double ch = dt / (mu0 * dx);
    double we = 0.0, wh = 0.0, wh2 = 0.0;
    int finite = 1;
    double dvol;
    if (s->p.ndim == 1) {
        const int64_t nz = s->nz;
        const double *ex = s->f[EX], *hy = s->f[HY];
        dvol = dx;
        for (int64_t k = 0; k <= nz; ++k) { we += ex[k] * ex[k]; finite &= isfinite(ex[k]); }
        for (int64_t k = 0; k < nz; ++k) {
            double hn = hy[k] - ch * (ex[k + 1] - ex[k]);
            wh += hy[k] * hn;
            wh2 += hy[k] * hy[k];
            finite &= isfinite(hy[k]);
        }
    } else if (s->p.ndim == 2) {
        const int64_t nx = s->nx, ny = s->ny;
        const double *ez = s->f[EZ], *hx = s->f[HX], *hy = s->f[HY];
        dvol = dx * dx;
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double e = ez[ID2(i, j)];
                double dEy = (j + 1 < ny ? ez[ID2(i, j + 1)] : 0.0) - e;
                double dEx = (i + 1 < nx ? ez[ID2(i + 1, j)] : 0.0) - e;
                double hxn = hx[ID2(i, j)] - ch * dEy, hyn = hy[ID2(i, j)] + ch * dEx;
                we += e * e;
                wh += hx[ID2(i, j)] * hxn + hy[ID2(i, j)] * hyn;
                wh2 += hx[ID2(i, j)] * hx[ID2(i, j)] + hy[ID2(i, j)] * hy[ID2(i, j)];
                finite &= isfinite(e) && isfinite(hx[ID2(i, j)]) && isfinite(hy[ID2(i, j)]);
            }
    } else {
        const int64_t nx = s->nx, ny = s->ny, nz = s->nz;
        const double *ex = s->f[EX], *ey = s->f[EY], *ez = s->f[EZ];
        const double *hx = s->f[HX], *hy = s->f[HY], *hz = s->f[HZ];
        dvol = dx * dx * dx;
#define EV(arr, i, j, k) (((i) < nx && (j) < ny && (k) < nz) ? arr[ID3(i, j, k)] : 0.0)
        for (int64_t k = 0; k < nz; ++k)
            for (int64_t j = 0; j < ny; ++j)
                for (int64_t i = 0; i < nx; ++i) {
                    int64_t c = ID3(i, j, k);
                    double hxn = hx[c] - ch * ((EV(ez, i, j + 1, k) - ez[c]) - (EV(ey, i, j, k + 1) - ey[c]));
                    double hyn = hy[c] - ch * ((EV(ex, i, j, k + 1) - ex[c]) - (EV(ez, i + 1, j, k) - ez[c]));
                    double hzn = hz[c] - ch * ((EV(ey, i + 1, j, k) - ey[c]) - (EV(ex, i, j + 1, k) - ex[c]));
                    we += ex[c] * ex[c] + ey[c] * ey[c] + ez[c] * ez[c];
                    wh += hx[c] * hxn + hy[c] * hyn + hz[c] * hzn;
                    wh2 += hx[c] * hx[c] + hy[c] * hy[c] + hz[c] * hz[c];
                    finite &= isfinite(ex[c]) && isfinite(ey[c]) && isfinite(ez[c]) && isfinite(hx[c]) &&
                              isfinite(hy[c]) && isfinite(hz[c]);
                }
#undef EV
    }
    double num = 0.0, nmax = 0.0, nabs = 0.0;
    for (int64_t q = 0; q < s->nslots; ++q) {
        const double *row = s->df + q * s->nnode;
        double c = 0.0;
        for (int64_t j = 0; j < s->nnode; ++j) {
            c += row[j] * s->dV[j];
            nabs += fabs(row[j]) * s->dV[j];
            finite &= isfinite(row[j]);
        }
        num += c;
        if (fabs(c) > nmax) nmax = fabs(c);
    }
    for (int q = 0; q < 12; ++q)
        if (s->psi[q])
            for (int64_t c = 0; c < s->ncell; ++c) finite &= isfinite(s->psi[q][c]);
    out[0] = (0.5 * OR_EPS0 * we + 0.5 * mu0 * wh) * dvol;
    out[1] = num;
    out[2] = nmax;
    out[3] = nabs;
    out[4] = finite ? 1.0 : 0.0;
    out[5] = (0.5 * OR_EPS0 * we + 0.5 * mu0 * wh2) * dvol;
}

/* ------------------------------------------------- 0-D driven kinetic cell */

/* One plasma cell of density n driven by a prescribed E^m, m = 0..nsteps-1,
 * with the same Sec. 5.2 update: returns J^{m+1/2} for every step and the
 * final delta f row.  Used to check the update against closed forms. */
void or_kinetic_drive(const or_params *p, double dt, double density, const double *E, int64_t nsteps,
                      double *J_out, double *df_out, double *g_out)
{
    const int64_t nn = or_nnode_of(p);
    double *v = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * nn);
    double *f0 = malloc(sizeof(double) * nn), *f0p = malloc(sizeof(double) * nn);
    double *nu = malloc(sizeof(double) * nn), *dV = malloc(sizeof(double) * nn);
    double *al = malloc(sizeof(double) * nn), *be = malloc(sizeof(double) * nn);
    or_vtables(p, dt, v, w, f0, f0p, nu, dV, al, be);
    double *row = (double *)calloc((size_t)nn, sizeof(double));
    double *g = (double *)calloc((size_t)nn, sizeof(double));
    double *scratch = (double *)malloc(sizeof(double) * 3 * nn);
    for (int64_t m = 0; m < nsteps; ++m) {
        if (p->evolve_f0) {
            evolve_row(p, dt, v, f0, f0p, nu, al, w, density, E[m], row, g, scratch, scratch + nn, scratch + 2 * nn,
                       &J_out[m]);
            continue;
        }
        double J = 0.0;
        for (int64_t j = 0; j < nn; ++j) {
            row[j] = al[j] * row[j] + be[j] * density * E[m];
            J += w[j] * row[j];
        }
        J_out[m] = -OR_QE * J;
    }
    if (df_out) memcpy(df_out, row, sizeof(double) * nn);
    if (g_out) memcpy(g_out, g, sizeof(double) * nn);
    free(v); free(w); free(f0); free(f0p); free(nu); free(dV); free(al); free(be); free(row); free(g); free(scratch);
}

/* ------------------------------------------------------------ Poynting flux */

/* Electromagnetic power out of an axis-aligned box, S = E x H, at time n:
 * E^n on the E-node planes that bound the box, H time-centred at n -- the mean
 * of the stored H^{n-1/2} and of H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n (vacuum
 * curl) -- and averaged in space onto the plane from the two neighbouring H
 * planes (an H plane outside the grid counts as 0).
 * box = {i0, i1, j0, j1, k0, k1}: the faces are the E-node planes i0, i1 (x),
 * j0, j1 (y), k0, k1 (z), each summed over the cell indices [lo, hi) of the
 * other two axes and weighted by the face element (dx^2 in 3-D, dx in 2-D, 1
 * in 1-D).  1-D uses the z faces k0, k1 (Ex Hy); 2-D TMz the x and y faces.
 * out[0..5] = power through the faces x0, x1, y0, y1, z0, z1 along +axis;
 * out[6] = net outward power = x1 - x0 + y1 - y0 + z1 - z0. */
void or_poynting(const or_sim *s, const int64_t *box, double *out)
{
    const int64_t nx = s->nx, ny = s->ny, nz = s->nz;
    const double mu0 = 1.0 / (OR_EPS0 * OR_C0 * OR_C0);
    const double ch = s->dt / (mu0 * s->p.dx);
    for (int q = 0; q < 7; ++q) out[q] = 0.0;
    if (s->p.ndim == 1) {
        const double *ex = s->f[EX], *hy = s->f[HY];
        for (int f = 0; f < 2; ++f) {
            const int64_t k = box[4 + f];
            double hb = 0.0;   /* time-centred Hy averaged onto node k */
            for (int64_t kk = k - 1; kk <= k; ++kk)
                if (kk >= 0 && kk < nz) hb += 0.5 * (hy[kk] - 0.5 * ch * (ex[kk + 1] - ex[kk]));
            out[4 + f] = ex[k] * hb;
        }
    } else if (s->p.ndim == 2) {
        const double *ez = s->f[EZ], *hx = s->f[HX], *hy = s->f[HY];
#define EZ2(i, j) ((i) < nx && (j) < ny ? ez[(j) * nx + (i)] : 0.0)
        /* time-centred H at its own position, 0 outside the grid */
#define HXT(i, j) ((i) >= 0 && (j) >= 0 && (i) < nx && (j) < ny ? hx[(j) * nx + (i)] - 0.5 * ch * (EZ2(i, (j) + 1) - EZ2(i, j)) : 0.0)
#define HYT(i, j) ((i) >= 0 && (j) >= 0 && (i) < nx && (j) < ny ? hy[(j) * nx + (i)] + 0.5 * ch * (EZ2((i) + 1, j) - EZ2(i, j)) : 0.0)
        const double dA = s->p.dx;
        for (int f = 0; f < 2; ++f) {
            const int64_t i = box[f];
            double acc = 0.0;
            for (int64_t j = box[2]; j < box[3]; ++j)   /* S_x = -Ez Hy */
                acc += -EZ2(i, j) * 0.5 * (HYT(i - 1, j) + HYT(i, j));
            out[f] = acc * dA;
        }
        for (int f = 0; f < 2; ++f) {
            const int64_t j = box[2 + f];
            double acc = 0.0;
            for (int64_t i = box[0]; i < box[1]; ++i)   /* S_y = Ez Hx */
                acc += EZ2(i, j) * 0.5 * (HXT(i, j - 1) + HXT(i, j));
            out[2 + f] = acc * dA;
        }
#undef EZ2
#undef HXT
#undef HYT
    } else {
        const double *ex = s->f[EX], *ey = s->f[EY], *ez = s->f[EZ];
        const double *hx = s->f[HX], *hy = s->f[HY], *hz = s->f[HZ];
#define E3(a, i, j, k) ((i) < nx && (j) < ny && (k) < nz ? (a)[((k) * ny + (j)) * nx + (i)] : 0.0)
#define IN3(i, j, k) ((i) >= 0 && (j) >= 0 && (k) >= 0 && (i) < nx && (j) < ny && (k) < nz)
#define HXT(i, j, k) (IN3(i, j, k) ? hx[((k) * ny + (j)) * nx + (i)] - 0.5 * ch * ((E3(ez, i, (j) + 1, k) - E3(ez, i, j, k)) - (E3(ey, i, j, (k) + 1) - E3(ey, i, j, k))) : 0.0)
#define HYT(i, j, k) (IN3(i, j, k) ? hy[((k) * ny + (j)) * nx + (i)] - 0.5 * ch * ((E3(ex, i, j, (k) + 1) - E3(ex, i, j, k)) - (E3(ez, (i) + 1, j, k) - E3(ez, i, j, k))) : 0.0)
#define HZT(i, j, k) (IN3(i, j, k) ? hz[((k) * ny + (j)) * nx + (i)] - 0.5 * ch * ((E3(ey, (i) + 1, j, k) - E3(ey, i, j, k)) - (E3(ex, i, (j) + 1, k) - E3(ex, i, j, k))) : 0.0)
        const double dA = s->p.dx * s->p.dx;
        for (int f = 0; f < 2; ++f) {   /* S_x = Ey Hz - Ez Hy */
            const int64_t i = box[f];
            double acc = 0.0;
            for (int64_t k = box[4]; k < box[5]; ++k)
                for (int64_t j = box[2]; j < box[3]; ++j)
                    acc += E3(ey, i, j, k) * 0.5 * (HZT(i - 1, j, k) + HZT(i, j, k)) -
                           E3(ez, i, j, k) * 0.5 * (HYT(i - 1, j, k) + HYT(i, j, k));
            out[f] = acc * dA;
        }
        for (int f = 0; f < 2; ++f) {   /* S_y = Ez Hx - Ex Hz */
            const int64_t j = box[2 + f];
            double acc = 0.0;
            for (int64_t k = box[4]; k < box[5]; ++k)
                for (int64_t i = box[0]; i < box[1]; ++i)
                    acc += E3(ez, i, j, k) * 0.5 * (HXT(i, j - 1, k) + HXT(i, j, k)) -
                           E3(ex, i, j, k) * 0.5 * (HZT(i, j - 1, k) + HZT(i, j, k));
            out[2 + f] = acc * dA;
        }
        for (int f = 0; f < 2; ++f) {   /* S_z = Ex Hy - Ey Hx */
            const int64_t k = box[4 + f];
            double acc = 0.0;
            for (int64_t j = box[2]; j < box[3]; ++j)
                for (int64_t i = box[0]; i < box[1]; ++i)
                    acc += E3(ex, i, j, k) * 0.5 * (HYT(i, j, k - 1) + HYT(i, j, k)) -
                           E3(ey, i, j, k) * 0.5 * (HXT(i, j, k - 1) + HXT(i, j, k));
            out[4 + f] = acc * dA;
        }
#undef E3
#undef IN3
#undef HXT
#undef HYT
#undef HZT
    }
    out[6] = out[1] - out[0] + out[3] - out[2] + out[5] - out[4];
}
