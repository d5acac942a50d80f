/*
 * grpic_oracle.c -- plain, slow FP64 CPU oracle of one GRPIC time step as
 * defined in Chen, Luepker & Yuan, "Introducing APERTURE: a GPU-based general
 * relativistic particle-in-cell simulation framework" (arXiv:2503.04558).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
 * and the cpu_baseline / reference leg of bench.py may load this library.  It
 * shares no source with the CUDA path (no headers, no helpers, no tables) and
 * the CUDA path never calls it.
 *
 * Every routine takes the paper's steps in the paper's order and notation with
 * plain loops; no blocking, fusion or reordering.  Built with
 * -O2 -ffp-contract=off.  Where the paper is silent, garbled or inconsistent
 * the adopted reading is named in the comment:
 *   - field corrector prefactor is dt, not dt/2 (Eq. fld-corrector with
 *     alpha+beta = 1; "alpha = beta = 1/2 is Heun's method");
 *   - E_phi's shift term carries the 1/2 of the two-point average (Eq. auxE);
 *   - the rotating Wald B^phi is the printed closed form (Eq. wald-solution-ks);
 *   - J^phi = +q (dphi/dt) <S> / dV (Eq. j-phi-deposit; sign and volume fixed
 *     so that the 3-current is a vector);
 *   - dphi = 1 for all phi integrals (2D axisymmetric cells);
 *   - edge lengths are coordinate extents: primal r_{i+1}-r_i for the B update,
 *     dual r_{i+1/2}-r_{i-1/2} for the D update (App. B);
 *   - CIC shape in logical (x1 = ln(r/r_in)/dx1, x2 = theta/dtheta) space;
 *   - axis reflection theta -> -theta, u_theta -> -u_theta (Sec. 2.1 BCs);
 *   - the first step of the Strang split is a full Boris step at fields n
 *     (bundled convention, Sec. 2.2 and Fig. stepping).
 *
 * Parity pins: see tests/test_oracle_*.py; every exported function here is
 * pinned by at least one test against something other than itself.  The
 * outer absorbing layer is pinned by its job (Sec. 2.1: fields damped to
 * zero at the outer boundary): an outgoing pulse is sent back by less than a
 * stated fraction and the layer's energy drains monotonically, against the
 * same run on an extended grid; its profile f <- f (1 - d_max s^3) over the
 * last damp_cells columns is a reading (the paper gives no profile), checked
 * entry by entry at each component's staggered column.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads for the timed CPU baseline (orc_set_threads; default 1, the
 * setting of every parity run).  With more than one thread the particle loop
 * of orc_push_deposit splits the particles into contiguous chunks, each
 * depositing into its own current arrays, summed in thread order at the end
 * (so J differs from the one-thread run only by the order of additions); the
 * field update's row loops write disjoint entries and give the same result
 * bit for bit.  Without OpenMP support in the compiler the pragmas are
 * ignored and everything runs on one thread. */
static int orc_nthreads = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    orc_nthreads = n < 1 ? 1 : n;
#else
    (void)n;
    orc_nthreads = 1;
#endif
    return orc_nthreads;
}

#define ORC_OK 0
#define ORC_ERANGE 4
#define ORC_ENAN 5
#define ORC_DEAD 0x80000000u

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Run configuration (grid of Sec. 2.1 / Fig. Yee, solver settings Sec. 2).  */
/* Field arrays are (nth+1) rows x ld columns, row j = theta index, column   */
/* c = i + ng where i is the r index (integer or half-integer location).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nr, nth, ng, ld;
    double a, r_in, r_out, dx1, dth;
    double dt, beta_s;
    int n_fld_iter, n_push_iter;
    int damp_cells;
    double damp_max;
    double qm[4];      /* q/m per species                                    */
    double qw[4];      /* deposited macro charge q*w per species             */
    int massive[4];    /* epsilon in u^0 (1 massive, 0 photon)               */
    int pusher;        /* momentum update: 0 generalized Boris, 1 Vay in the  */
                       /* FIDO frame (Sec. 2.2)                              */
    int shape;         /* particle shape (Sec. 2.3): 1 cloud in cell, 3 the  */
                       /* third-order (cubic B-) spline                      */
    int radiation;     /* 2D photon emission and pair conversion (Sec. 4)    */
    int injection;     /* pair injection of the plasma-filled Wald run       */
    double gamma_thr, eps_ph, tau;   /* emission threshold, photon energy,   */
                                     /* conversion opacity                   */
    double sigma_thr, eps_db;        /* injection thresholds                 */
    uint64_t seed;                   /* Philox key                           */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* Kerr-Schild 3+1 metric, App. A (Eqs. ks-coefficients, ks-variables,       */
/* gamma-inverse, ks-alpha-beta) with analytic r and theta derivatives.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double alpha, beta;                     /* lapse, shift beta^r            */
    double g_rr, g_rp, g_thth, g_pp;        /* gamma_ij                        */
    double gi_rr, gi_rp, gi_thth, gi_pp;    /* gamma^ij                        */
    double sqrtg;                           /* sqrt(det gamma_ij)              */
    double da[2], db[2];                    /* d_r, d_theta of alpha, beta^r   */
    double dgi_rr[2], dgi_rp[2], dgi_thth[2], dgi_pp[2];
} orc_metric;

static void metric_at(double a, double r, double th, orc_metric *m)
{
    double s = sin(th), c = cos(th);
    double rho2 = r * r + a * a * c * c;
    double Delta = r * r + a * a - 2.0 * r;
    double Sigma = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s * s;
    double z = 2.0 * r / rho2;

    /* Eq. ks-coefficients: gamma_ij = g_ij */
    m->g_rr = 1.0 + z;
    m->g_thth = rho2;
    m->g_pp = Sigma * s * s / rho2;
    m->g_rp = -a * s * s * (1.0 + z);
    /* Eq. gamma-inverse */
    m->gi_rr = (a * a + r * r) / rho2 - 2.0 * r / (rho2 + 2.0 * r);
    m->gi_rp = a / rho2;
    m->gi_thth = 1.0 / rho2;
    m->gi_pp = 1.0 / (rho2 * s * s);
    /* Eq. ks-alpha-beta */
    m->alpha = 1.0 / sqrt(1.0 + z);
    m->beta = z / (1.0 + z);
    /* sqrt(gamma) from its definition, the determinant of gamma_ij */
    m->sqrtg = sqrt(m->g_thth * (m->g_rr * m->g_pp - m->g_rp * m->g_rp));

    /* analytic derivatives, index 0 = d/dr, 1 = d/dtheta */
    double drho2[2] = {2.0 * r, -2.0 * a * a * c * s};
    double rho4 = rho2 * rho2;
    double dz[2];
    dz[0] = 2.0 / rho2 - 2.0 * r * drho2[0] / rho4;
    dz[1] = -2.0 * r * drho2[1] / rho4;
    for (int k = 0; k < 2; ++k) {
        double opz = 1.0 + z;
        m->da[k] = -0.5 * pow(opz, -1.5) * dz[k];
        m->db[k] = dz[k] / (opz * opz);
        m->dgi_rp[k] = -a * drho2[k] / rho4;
        m->dgi_thth[k] = -drho2[k] / rho4;
    }
    /* gamma^rr = (a^2+r^2)/rho^2 - z/(1+z) */
    m->dgi_rr[0] = 2.0 * r / rho2 - (a * a + r * r) * drho2[0] / rho4 - m->db[0];
    m->dgi_rr[1] = -(a * a + r * r) * drho2[1] / rho4 - m->db[1];
    /* gamma^phiphi = 1/(rho^2 sin^2) */
    m->dgi_pp[0] = -drho2[0] / (rho4 * s * s);
    m->dgi_pp[1] = -(drho2[1] * s * s + rho2 * 2.0 * s * c) / (rho4 * s * s * s * s);
}

/* out[0..29]: alpha, beta, g_rr, g_rp, g_thth, g_pp, gi_rr, gi_rp, gi_thth,
 * gi_pp, sqrtg, da[2], db[2], dgi_rr[2], dgi_rp[2], dgi_thth[2], dgi_pp[2] */
void orc_metric_eval(double a, double r, double th, double *out)
{
    orc_metric m;
    metric_at(a, r, th, &m);
    double v[23] = {m.alpha, m.beta, m.g_rr, m.g_rp, m.g_thth, m.g_pp,
                    m.gi_rr, m.gi_rp, m.gi_thth, m.gi_pp, m.sqrtg,
                    m.da[0], m.da[1], m.db[0], m.db[1],
                    m.dgi_rr[0], m.dgi_rr[1], m.dgi_rp[0], m.dgi_rp[1],
                    m.dgi_thth[0], m.dgi_thth[1], m.dgi_pp[0], m.dgi_pp[1]};
    memcpy(out, v, sizeof v);
}

/* ------------------------------------------------------------------------ */
/* Analytic initial fields, Sec. 3.3 and App. C.                             */
/* kind 0: rotating Wald (Eqs. wald-vector-potential, wald-solution-ks)      */
/* kind 1: non-rotating Wald in the spinning metric (Eq.                     */
/*         vacuum-nonrotating-wald: E_i = 0, A_phi = B0 gamma_phiphi / 2)    */
/* kind 2: monopole (App. C)   kind 3: split monopole = sgn(cos th) monopole */
/* Returned: A_t, A_phi, E_i (covariant), sqrt(gamma) B^i (contravariant).   */
/* ------------------------------------------------------------------------ */
static void closed_fields(int kind, double a, double B0, double r, double th,
                          double *At, double *Aph, double E[3], double sgB[3])
{
    double s = sin(th), c = cos(th);
    double rho2 = r * r + a * a * c * c, rho4 = rho2 * rho2;
    double Delta = r * r + a * a - 2.0 * r;
    if (kind == 0) {
        *At = B0 * (a * r * (1.0 + c * c) / rho2 - a);
        *Aph = B0 * 0.5 * s * s * (r * r + a * a - 2.0 * a * a * r * (1.0 + c * c) / rho2);
        sgB[0] = B0 * (Delta + 2.0 * r * (r * r * r * r - a * a * a * a) / rho4) * s * c;
        sgB[1] = -B0 * (r + a * a * (1.0 + c * c) * (2.0 * r * r - rho2) / rho4) * s * s;
        sgB[2] = -B0 * (2.0 * a * r * (a * a - r * r) / rho4 - a) * s * c;
        E[0] = B0 * a * (1.0 + c * c) * (a * a * c * c - r * r) / rho4;
        E[1] = B0 * 2.0 * a * r * (a * a - r * r) * s * c / rho4;
        E[2] = 0.0;
    } else if (kind == 1) {
        orc_metric m;
        metric_at(a, r, th, &m);
        /* gamma_phiphi = Sigma sin^2 / rho^2; derivatives written out */
        double Sigma = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s * s;
        double dS_dr = 4.0 * r * (r * r + a * a) - a * a * (2.0 * r - 2.0) * s * s;
        double dS_dth = -a * a * Delta * 2.0 * s * c;
        double drho2_dr = 2.0 * r, drho2_dth = -2.0 * a * a * c * s;
        double gpp_r = (dS_dr * s * s * rho2 - Sigma * s * s * drho2_dr) / rho4;
        double gpp_th = ((dS_dth * s * s + Sigma * 2.0 * s * c) * rho2 - Sigma * s * s * drho2_dth) / rho4;
        *At = 0.0;
        *Aph = 0.5 * B0 * m.g_pp;
        sgB[0] = 0.5 * B0 * gpp_th;
        sgB[1] = -0.5 * B0 * gpp_r;
        sgB[2] = 0.0;
        E[0] = E[1] = E[2] = 0.0;
    } else {
        double sg = 1.0;
        if (kind == 3) sg = (c > 0.0) ? 1.0 : ((c < 0.0) ? -1.0 : 0.0);
        *At = sg * B0 * a * c / rho2;
        *Aph = -sg * B0 * c * (r * r + a * a) / rho2;
        sgB[0] = sg * B0 * (a * a + r * r) * (r * r - a * a * c * c) * s / rho4;
        sgB[1] = -sg * B0 * 2.0 * a * a * r * s * s * c / rho4;
        sgB[2] = sg * B0 * a * (r * r - a * a * c * c) * s / rho4;
        E[0] = -sg * B0 * 2.0 * a * r * c / rho4;
        E[1] = -sg * B0 * a * (r * r - a * a * c * c) * s / rho4;
        E[2] = 0.0;
    }
}

/* D^j = gamma^{ji} (E_i - e_ikl beta^k B^l) / alpha, from Eq. E-H-B-D solved
 * for D.  With beta = (beta^r, 0, 0): e_{theta r phi} = -sqrt(gamma),
 * e_{phi r theta} = +sqrt(gamma). */
static void closed_D(int kind, double a, double B0, double r, double th, double D[3], double Bup[3])
{
    orc_metric m;
    double At, Aph, E[3], sgB[3];
    metric_at(a, r, th, &m);
    closed_fields(kind, a, B0, r, th, &At, &Aph, E, sgB);
    double Ep_r = E[0];
    double Ep_th = E[1] + m.beta * sgB[2];
    double Ep_ph = E[2] - m.beta * sgB[1];
    D[0] = (m.gi_rr * Ep_r + m.gi_rp * Ep_ph) / m.alpha;
    D[1] = m.gi_thth * Ep_th / m.alpha;
    D[2] = (m.gi_rp * Ep_r + m.gi_pp * Ep_ph) / m.alpha;
    for (int k = 0; k < 3; ++k) Bup[k] = sgB[k] / m.sqrtg;
}

/* out[0..9]: At, Aph, E_r, E_th, E_ph, sg*B^r, sg*B^th, sg*B^ph, then D^r..D^ph
 * follow in out[10..12] and B^r..B^ph in out[13..15]. */
void orc_closed_fields(int kind, double a, double B0, double r, double th, double *out)
{
    double At, Aph, E[3], sgB[3], D[3], Bu[3];
    closed_fields(kind, a, B0, r, th, &At, &Aph, E, sgB);
    closed_D(kind, a, B0, r, th, D, Bu);
    double v[16] = {At, Aph, E[0], E[1], E[2], sgB[0], sgB[1], sgB[2], 0, 0, D[0], D[1], D[2], Bu[0], Bu[1], Bu[2]};
    memcpy(out, v, sizeof v);
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre quadrature (Sec. 2.1: "a simple 10-point Gauss            */
/* quadrature"); nodes by Newton's method on the Legendre recurrence.        */
/* ------------------------------------------------------------------------ */
#define NGL 10
static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    int n = NGL;
    for (int k = 0; k < n; ++k) {
        double x = cos(M_PI * (k + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = x;
        for (int l = 2; l <= n; ++l) {
            double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[k] = x;
        gl_w[k] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

void orc_gauss_legendre(double *x, double *w)
{
    gl_init();
    memcpy(x, gl_x, sizeof gl_x);
    memcpy(w, gl_w, sizeof gl_w);
}

static double sqrtg_at(double a, double r, double th)
{
    orc_metric m;
    metric_at(a, r, th, &m);
    return m.sqrtg;
}

/* integral of sqrt(gamma) over theta in [t0,t1] at fixed r (dphi = 1) */
static double int_th(double a, double r, double t0, double t1)
{
    gl_init();
    double h = 0.5 * (t1 - t0), mid = 0.5 * (t1 + t0), s = 0.0;
    for (int k = 0; k < NGL; ++k) s += gl_w[k] * sqrtg_at(a, r, mid + h * gl_x[k]);
    return h * s;
}
/* integral over r in [r0,r1] at fixed theta */
static double int_r(double a, double r0, double r1, double th)
{
    gl_init();
    double h = 0.5 * (r1 - r0), mid = 0.5 * (r1 + r0), s = 0.0;
    for (int k = 0; k < NGL; ++k) s += gl_w[k] * sqrtg_at(a, mid + h * gl_x[k], th);
    return h * s;
}
/* 10 x 10 point rule over [r0,r1] x [t0,t1] */
static double int_rth(double a, double r0, double r1, double t0, double t1)
{
    gl_init();
    double hr = 0.5 * (r1 - r0), mr = 0.5 * (r1 + r0);
    double ht = 0.5 * (t1 - t0), mt = 0.5 * (t1 + t0), s = 0.0;
    for (int k = 0; k < NGL; ++k)
        for (int l = 0; l < NGL; ++l)
            s += gl_w[k] * gl_w[l] * sqrtg_at(a, mr + hr * gl_x[k], mt + ht * gl_x[l]);
    return hr * ht * s;
}

/* ------------------------------------------------------------------------ */
/* Grid geometry: log-r x theta, Fig. Yee staggering                        */
/*   D^r, B^th, J^r  at (i+1/2, j)   D^th, B^r, J^th at (i, j+1/2)          */
/*   D^ph, J^ph, rho at (i, j)       B^ph            at (i+1/2, j+1/2)      */
/* ------------------------------------------------------------------------ */
static double r_of(const orc_cfg *c, double x1) { return c->r_in * exp(x1 * c->dx1); }

enum { LOC_DR = 0, LOC_DT, LOC_DP, LOC_BR, LOC_BT, LOC_BP };
/* stagger (in r, in theta) of each location, in cells */
static const double STAG_R[6] = {0.5, 0.0, 0.0, 0.0, 0.5, 0.5};
static const double STAG_T[6] = {0.0, 0.5, 0.0, 0.5, 0.0, 0.5};

typedef struct {
    orc_cfg c;
    int n;            /* (nth+1)*ld */
    /* area elements, Eq. area-element; A^D_i at D^i locations, A^B_i at B^i */
    double *AD[3], *AB[3];
    /* point metric products at every location (Eqs. auxE, auxH) */
    double *ag_rr[6], *ag_rp[6], *ag_thth[6], *ag_pp[6], *sgb[6];
    double *dr_prim, *dr_dual;   /* per column */
} orc_geom;

#define IDX(c, i, j) ((j) * (c)->ld + (i) + (c)->ng)

static void geom_free(orc_geom *g)
{
    for (int k = 0; k < 3; ++k) { free(g->AD[k]); free(g->AB[k]); }
    for (int k = 0; k < 6; ++k) { free(g->ag_rr[k]); free(g->ag_rp[k]); free(g->ag_thth[k]); free(g->ag_pp[k]); free(g->sgb[k]); }
    free(g->dr_prim); free(g->dr_dual);
}

static void geom_build(const orc_cfg *c, orc_geom *g)
{
    memset(g, 0, sizeof *g);
    g->c = *c;
    g->n = (c->nth + 1) * c->ld;
    for (int k = 0; k < 3; ++k) {
        g->AD[k] = calloc(g->n, sizeof(double));
        g->AB[k] = calloc(g->n, sizeof(double));
    }
    for (int k = 0; k < 6; ++k) {
        g->ag_rr[k] = calloc(g->n, sizeof(double));
        g->ag_rp[k] = calloc(g->n, sizeof(double));
        g->ag_thth[k] = calloc(g->n, sizeof(double));
        g->ag_pp[k] = calloc(g->n, sizeof(double));
        g->sgb[k] = calloc(g->n, sizeof(double));
    }
    g->dr_prim = calloc(c->ld, sizeof(double));
    g->dr_dual = calloc(c->ld, sizeof(double));
    double dth = c->dth, a = c->a;
    for (int i = -c->ng; i < c->ld - c->ng; ++i) {
        g->dr_prim[i + c->ng] = r_of(c, i + 1.0) - r_of(c, i);
        g->dr_dual[i + c->ng] = r_of(c, i + 0.5) - r_of(c, i - 0.5);
    }
    for (int j = 0; j <= c->nth; ++j) {
        double tlo = (j - 0.5) * dth, thi = (j + 0.5) * dth; /* dual theta range */
        if (tlo < 0.0) tlo = 0.0;
        if (thi > M_PI) thi = M_PI;
        for (int i = -c->ng; i < c->ld - c->ng; ++i) {
            int q = IDX(c, i, j);
            double ri = r_of(c, i), rh = r_of(c, i + 0.5);
            double rml = r_of(c, i - 0.5), rp1 = r_of(c, i + 1.0);
            /* D^r face: r = r_{i+1/2}, theta in dual range */
            g->AD[0][q] = int_th(a, rh, tlo, thi);
            /* D^phi face: dual r and theta ranges */
            g->AD[2][q] = int_rth(a, rml, rh, tlo, thi);
            /* B^th face: theta = theta_j, primal r range */
            g->AB[1][q] = int_r(a, ri, rp1, j * dth);
            if (j < c->nth) {
                /* D^th face: theta = theta_{j+1/2}, dual r range */
                g->AD[1][q] = int_r(a, rml, rh, (j + 0.5) * dth);
                /* B^r face: r = r_i, primal theta range */
                g->AB[0][q] = int_th(a, ri, j * dth, (j + 1) * dth);
                /* B^ph face: primal r and theta ranges */
                g->AB[2][q] = int_rth(a, ri, rp1, j * dth, (j + 1) * dth);
            }
            for (int L = 0; L < 6; ++L) {
                if (STAG_T[L] > 0.0 && j == c->nth) continue;
                orc_metric m;
                metric_at(a, r_of(c, i + STAG_R[L]), (j + STAG_T[L]) * dth, &m);
                g->ag_rr[L][q] = m.alpha * m.g_rr;
                g->ag_rp[L][q] = m.alpha * m.g_rp;
                g->ag_thth[L][q] = m.alpha * m.g_thth;
                g->ag_pp[L][q] = m.alpha * m.g_pp;
                g->sgb[L][q] = m.sqrtg * m.beta;
            }
        }
    }
}

/* The tables depend only on the grid; keep the last one (a plain cache, the
 * values are identical to a fresh build). */
static orc_geom g_cache;
static int g_cache_ok = 0;
static const orc_geom *geom_get(const orc_cfg *c)
{
    if (g_cache_ok && g_cache.c.nr == c->nr && g_cache.c.nth == c->nth && g_cache.c.ng == c->ng &&
        g_cache.c.ld == c->ld && g_cache.c.a == c->a && g_cache.c.r_in == c->r_in &&
        g_cache.c.r_out == c->r_out && g_cache.c.dx1 == c->dx1 && g_cache.c.dth == c->dth) {
        g_cache.c = *c;
        return &g_cache;
    }
    if (g_cache_ok) geom_free(&g_cache);
    geom_build(c, &g_cache);
    g_cache_ok = 1;
    return &g_cache;
}

/* Export the area tables (for pins P14 and parity of the tables). */
void orc_areas(const orc_cfg *c, double *AD0, double *AD1, double *AD2, double *AB0, double *AB1, double *AB2)
{
    const orc_geom *g = geom_get(c);
    size_t bytes = (size_t)g->n * sizeof(double);
    memcpy(AD0, g->AD[0], bytes); memcpy(AD1, g->AD[1], bytes); memcpy(AD2, g->AD[2], bytes);
    memcpy(AB0, g->AB[0], bytes); memcpy(AB1, g->AB[1], bytes); memcpy(AB2, g->AB[2], bytes);
}

/* ------------------------------------------------------------------------ */
/* Field boundary conditions, Sec. 2.1: axis D^phi = B^theta = 0; inner     */
/* guard cells copy the first physical cell (zero derivative); the outer     */
/* guard cells are filled the same way (the damping layer lies inside).      */
/* ------------------------------------------------------------------------ */
static void apply_bc(const orc_cfg *c, double *D[3], double *B[3])
{
    double *half_r[3] = {D[0], B[1], B[2]};   /* last physical i = nr-1 */
    double *int_r[3] = {D[1], D[2], B[0]};    /* last physical i = nr   */
    for (int j = 0; j <= c->nth; ++j) {
        for (int k = 0; k < 3; ++k) {
            for (int i = -c->ng; i < 0; ++i) {
                half_r[k][IDX(c, i, j)] = half_r[k][IDX(c, 0, j)];
                int_r[k][IDX(c, i, j)] = int_r[k][IDX(c, 0, j)];
            }
            for (int i = c->nr; i < c->ld - c->ng; ++i) half_r[k][IDX(c, i, j)] = half_r[k][IDX(c, c->nr - 1, j)];
            for (int i = c->nr + 1; i < c->ld - c->ng; ++i) int_r[k][IDX(c, i, j)] = int_r[k][IDX(c, c->nr, j)];
        }
    }
    for (int i = -c->ng; i < c->ld - c->ng; ++i) {
        D[2][IDX(c, i, 0)] = 0.0;
        D[2][IDX(c, i, c->nth)] = 0.0;
        B[1][IDX(c, i, 0)] = 0.0;
        B[1][IDX(c, i, c->nth)] = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Initial fields (App. C): B^r, B^theta by Stokes' theorem on A_phi over    */
/* each primal face; B^phi as the face average of the closed form; D^j      */
/* pointwise from the closed-form E_i and B^l.                               */
/* ------------------------------------------------------------------------ */
static double Aphi_at(int kind, double a, double B0, double r, double th)
{
    double At, Aph, E[3], sgB[3];
    closed_fields(kind, a, B0, r, th, &At, &Aph, E, sgB);
    return Aph;
}

void orc_init_fields(const orc_cfg *c, int kind, double B0, double *D0, double *D1, double *D2,
                     double *B0r, double *B1, double *B2)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    double *D[3] = {D0, D1, D2}, *B[3] = {B0r, B1, B2};
    double a = c->a, dth = c->dth;
    for (int k = 0; k < 3; ++k) {
        memset(D[k], 0, sizeof(double) * g.n);
        memset(B[k], 0, sizeof(double) * g.n);
    }
    gl_init();
    for (int j = 0; j <= c->nth; ++j) {
        for (int i = -c->ng; i < c->ld - c->ng; ++i) {
            int q = IDX(c, i, j);
            double ri = r_of(c, i), rp1 = r_of(c, i + 1.0);
            if (j < c->nth) {
                /* B^r A^B_r = A_phi(r_i, th_{j+1}) - A_phi(r_i, th_j) */
                B[0][q] = (Aphi_at(kind, a, B0, ri, (j + 1) * dth) - Aphi_at(kind, a, B0, ri, j * dth)) / g.AB[0][q];
                /* B^ph A^B_ph = integral of sqrt(gamma) B^phi over the face */
                double hr = 0.5 * (rp1 - ri), mr = 0.5 * (rp1 + ri);
                double ht = 0.5 * dth, mt = (j + 0.5) * dth, s = 0.0;
                for (int kk = 0; kk < NGL; ++kk)
                    for (int l = 0; l < NGL; ++l) {
                        double At, Aph, E[3], sgB[3];
                        closed_fields(kind, a, B0, mr + hr * gl_x[kk], mt + ht * gl_x[l], &At, &Aph, E, sgB);
                        s += gl_w[kk] * gl_w[l] * sgB[2];
                    }
                B[2][q] = hr * ht * s / g.AB[2][q];
            }
            if (j > 0 && j < c->nth) {
                /* B^th A^B_th = -(A_phi(r_{i+1}, th_j) - A_phi(r_i, th_j)) */
                B[1][q] = -(Aphi_at(kind, a, B0, rp1, j * dth) - Aphi_at(kind, a, B0, ri, j * dth)) / g.AB[1][q];
            }
            double Dv[3], Bu[3];
            closed_D(kind, a, B0, r_of(c, i + 0.5), j * dth, Dv, Bu);
            D[0][q] = Dv[0];
            if (j < c->nth) {
                closed_D(kind, a, B0, r_of(c, i), (j + 0.5) * dth, Dv, Bu);
                D[1][q] = Dv[1];
            }
            if (j > 0 && j < c->nth) {
                closed_D(kind, a, B0, r_of(c, i), j * dth, Dv, Bu);
                D[2][q] = Dv[2];
            }
        }
    }
    apply_bc(c, D, B);
}

/* ------------------------------------------------------------------------ */
/* Auxiliary fields, Eqs. auxH and auxE (metric factors multiplied before   */
/* the two-point averages), and the circulations of Eqs. D-update and        */
/* B-update.  Evaluated over every index whose neighbours exist.             */
/* ------------------------------------------------------------------------ */
static void aux_fields(const orc_geom *g, double *const D[3], double *const B[3], double *E[3], double *H[3])
{
    const orc_cfg *c = &g->c;
    for (int k = 0; k < 3; ++k) {
        memset(E[k], 0, sizeof(double) * g->n);
        memset(H[k], 0, sizeof(double) * g->n);
    }
    int ilo = -c->ng + 1, ihi = c->ld - c->ng - 2;
#pragma omp parallel for schedule(static) num_threads(orc_nthreads) if (orc_nthreads > 1)
    for (int j = 0; j <= c->nth; ++j) {
        for (int i = ilo; i <= ihi; ++i) {
            int q = IDX(c, i, j), qm = IDX(c, i - 1, j), qp = IDX(c, i + 1, j);
            if (j < c->nth) {
                /* H_r at B^r location (i, j+1/2) */
                H[0][q] = g->ag_rr[LOC_BR][q] * B[0][q]
                        + 0.5 * (g->ag_rp[LOC_BP][q] * B[2][q] + g->ag_rp[LOC_BP][qm] * B[2][qm]);
                /* H_phi at B^phi location (i+1/2, j+1/2) */
                H[2][q] = g->ag_pp[LOC_BP][q] * B[2][q]
                        + 0.5 * (g->ag_rp[LOC_BR][q] * B[0][q] + g->ag_rp[LOC_BR][qp] * B[0][qp])
                        - 0.5 * (g->sgb[LOC_DT][q] * D[1][q] + g->sgb[LOC_DT][qp] * D[1][qp]);
                /* E_theta at D^th location (i, j+1/2) */
                E[1][q] = g->ag_thth[LOC_DT][q] * D[1][q]
                        - 0.5 * (g->sgb[LOC_BP][q] * B[2][q] + g->sgb[LOC_BP][qm] * B[2][qm]);
            }
            /* H_theta at B^th location (i+1/2, j) */
            H[1][q] = g->ag_thth[LOC_BT][q] * B[1][q]
                    + 0.5 * (g->sgb[LOC_DP][q] * D[2][q] + g->sgb[LOC_DP][qp] * D[2][qp]);
            /* E_r at D^r location (i+1/2, j) */
            E[0][q] = g->ag_rr[LOC_DR][q] * D[0][q]
                    + 0.5 * (g->ag_rp[LOC_DP][q] * D[2][q] + g->ag_rp[LOC_DP][qp] * D[2][qp]);
            /* E_phi at D^ph location (i, j); the shift term takes the 1/2 of the
             * two-point average like every other average in Eq. auxE */
            E[2][q] = g->ag_pp[LOC_DP][q] * D[2][q]
                    + 0.5 * (g->ag_rp[LOC_DR][q] * D[0][q] + g->ag_rp[LOC_DR][qm] * D[0][qm])
                    + 0.5 * (g->sgb[LOC_BT][q] * B[1][q] + g->sgb[LOC_BT][qm] * B[1][qm]);
        }
    }
}

/* C_H (into CD) and C_E (into CB) on the physical index ranges; dphi = 1 */
static void circulations(const orc_geom *g, double *E[3], double *H[3], double *CD[3], double *CB[3])
{
    const orc_cfg *c = &g->c;
    for (int k = 0; k < 3; ++k) {
        memset(CD[k], 0, sizeof(double) * g->n);
        memset(CB[k], 0, sizeof(double) * g->n);
    }
#pragma omp parallel for schedule(static) num_threads(orc_nthreads) if (orc_nthreads > 1)
    for (int j = 0; j <= c->nth; ++j) {
        for (int i = 0; i <= c->nr; ++i) {
            int q = IDX(c, i, j), qm = IDX(c, i - 1, j), qp = IDX(c, i + 1, j);
            int qjm = IDX(c, i, j - 1), qjp = IDX(c, i, j + 1);
            if (i < c->nr) {
                /* D^r (Eq. D-update; on the axis only the interior H_phi edge
                 * contributes, Eq. Dr-axis with the half-width face area) */
                double hp = (j < c->nth) ? H[2][q] : 0.0;
                double hm = (j > 0) ? H[2][qjm] : 0.0;
                CD[0][q] = (hp - hm) / g->AD[0][q];
            }
            if (j < c->nth) {
                /* D^theta */
                CD[1][q] = (H[2][qm] - H[2][q]) / g->AD[1][q];
                /* B^r (Eq. B-update) */
                CB[0][q] = -(E[2][qjp] - E[2][q]) / g->AB[0][q];
            }
            if (j > 0 && j < c->nth) {
                /* D^phi with dual edge lengths */
                CD[2][q] = ((H[1][q] - H[1][qm]) * c->dth + (H[0][qjm] - H[0][q]) * g->dr_dual[i + c->ng]) / g->AD[2][q];
                if (i < c->nr) /* B^theta (zero on the axis) */
                    CB[1][q] = -(E[2][q] - E[2][qp]) / g->AB[1][q];
            }
            if (i < c->nr && j < c->nth) {
                /* B^phi with primal edge lengths */
                CB[2][q] = -((E[1][qp] - E[1][q]) * c->dth + (E[0][q] - E[0][qjp]) * g->dr_prim[i + c->ng]) / g->AB[2][q];
            }
        }
    }
}

static int is_phys(const orc_cfg *c, int comp, int i, int j)
{
    /* comp 0..2 = D^r, D^th, D^ph, 3..5 = B^r, B^th, B^ph */
    int half_r = (comp == 0 || comp == 4 || comp == 5);
    int half_t = (comp == 1 || comp == 3 || comp == 5);
    if (i < 0) return 0;
    if (half_r ? (i > c->nr - 1) : (i > c->nr)) return 0;
    if (half_t ? (j > c->nth - 1) : (j > c->nth)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Field update n -> n+1, Eqs. fld-predictor and fld-corrector:             */
/*   predictor  X~ = X^n + dt (C(X^n) - J)                                   */
/*   corrector  X  = X^n + dt (alpha_s C(X^n) + beta_s C(X~)) - dt J,        */
/*              iterated n_fld_iter times, X~ <- latest iterate              */
/* J^r, J^th, J^ph are current densities (already divided by A^D).           */
/* Boundary conditions after every stage; outer damping once per step:       */
/*   f <- f (1 - damp_max s^3), s = depth into the last damp_cells cells.    */
/* ------------------------------------------------------------------------ */
void orc_field_update(const orc_cfg *c, double *D0, double *D1, double *D2, double *B0r, double *B1, double *B2,
                      const double *J0, const double *J1, const double *J2)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    int n = g.n;
    double *Dn[3] = {D0, D1, D2}, *Bn[3] = {B0r, B1, B2};
    const double *J[3] = {J0, J1, J2};
    double *E[3], *H[3], *CDn[3], *CBn[3], *CD[3], *CB[3], *Dt[3], *Bt[3];
    for (int k = 0; k < 3; ++k) {
        E[k] = malloc(n * sizeof(double)); H[k] = malloc(n * sizeof(double));
        CDn[k] = malloc(n * sizeof(double)); CBn[k] = malloc(n * sizeof(double));
        CD[k] = malloc(n * sizeof(double)); CB[k] = malloc(n * sizeof(double));
        Dt[k] = malloc(n * sizeof(double)); Bt[k] = malloc(n * sizeof(double));
    }
    double dt = c->dt, bs = c->beta_s, as = 1.0 - c->beta_s;

    aux_fields(&g, Dn, Bn, E, H);
    circulations(&g, E, H, CDn, CBn);
    /* predictor */
    for (int k = 0; k < 3; ++k) {
        memcpy(Dt[k], Dn[k], n * sizeof(double));
        memcpy(Bt[k], Bn[k], n * sizeof(double));
    }
#pragma omp parallel for schedule(static) num_threads(orc_nthreads) if (orc_nthreads > 1)
    for (int j = 0; j <= c->nth; ++j)
        for (int i = 0; i <= c->nr; ++i) {
            int q = IDX(c, i, j);
            for (int k = 0; k < 3; ++k) {
                if (is_phys(c, k, i, j)) Dt[k][q] = Dn[k][q] + (CDn[k][q] - J[k][q]) * dt;
                if (is_phys(c, 3 + k, i, j)) Bt[k][q] = Bn[k][q] + CBn[k][q] * dt;
            }
        }
    apply_bc(c, Dt, Bt);
    /* correctors */
    for (int it = 0; it < c->n_fld_iter; ++it) {
        aux_fields(&g, Dt, Bt, E, H);
        circulations(&g, E, H, CD, CB);
#pragma omp parallel for schedule(static) num_threads(orc_nthreads) if (orc_nthreads > 1)
        for (int j = 0; j <= c->nth; ++j)
            for (int i = 0; i <= c->nr; ++i) {
                int q = IDX(c, i, j);
                for (int k = 0; k < 3; ++k) {
                    if (is_phys(c, k, i, j)) Dt[k][q] = Dn[k][q] + dt * (as * CDn[k][q] + bs * CD[k][q]) - J[k][q] * dt;
                    if (is_phys(c, 3 + k, i, j)) Bt[k][q] = Bn[k][q] + dt * (as * CBn[k][q] + bs * CB[k][q]);
                }
            }
        apply_bc(c, Dt, Bt);
    }
    /* outer damping layer */
    if (c->damp_cells > 0 && c->damp_max > 0.0) {
        double x0 = c->nr - c->damp_cells;
        for (int j = 0; j <= c->nth; ++j)
            for (int i = 0; i <= c->nr; ++i) {
                int q = IDX(c, i, j);
                for (int comp = 0; comp < 6; ++comp) {
                    if (!is_phys(c, comp, i, j)) continue;
                    double x = i + ((comp == 0 || comp == 4 || comp == 5) ? 0.5 : 0.0);
                    double s = (x - x0) / c->damp_cells;
                    if (s <= 0.0) continue;
                    if (s > 1.0) s = 1.0;
                    double f = 1.0 - c->damp_max * s * s * s;
                    if (comp < 3) Dt[comp][q] *= f; else Bt[comp - 3][q] *= f;
                }
            }
        apply_bc(c, Dt, Bt);
    }
    for (int k = 0; k < 3; ++k) {
        memcpy(Dn[k], Dt[k], n * sizeof(double));
        memcpy(Bn[k], Bt[k], n * sizeof(double));
        free(E[k]); free(H[k]); free(CDn[k]); free(CBn[k]); free(CD[k]); free(CB[k]); free(Dt[k]); free(Bt[k]);
    }
}

/* circulations of the given fields, for pins (C_H into CD*, C_E into CB*) */
void orc_circulations(const orc_cfg *c, double *D0, double *D1, double *D2, double *B0r, double *B1, double *B2,
                      double *CD0, double *CD1, double *CD2, double *CB0, double *CB1, double *CB2)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    double *D[3] = {D0, D1, D2}, *B[3] = {B0r, B1, B2};
    double *CD[3] = {CD0, CD1, CD2}, *CB[3] = {CB0, CB1, CB2};
    double *E[3], *H[3];
    for (int k = 0; k < 3; ++k) { E[k] = malloc(g.n * sizeof(double)); H[k] = malloc(g.n * sizeof(double)); }
    aux_fields(&g, D, B, E, H);
    circulations(&g, E, H, CD, CB);
    for (int k = 0; k < 3; ++k) { free(E[k]); free(H[k]); }
}

/* ------------------------------------------------------------------------ */
/* Particle pusher, Sec. 2.2                                                 */
/* ------------------------------------------------------------------------ */

/* right-hand sides X^i, U_i of Eq. particle-eom without the Lorentz force;
 * y = (r, theta, phi, u_r, u_theta, u_phi); U_phi = 0 by axisymmetry */
static void geo_rhs(double a, double eps, const double y[6], double f[6])
{
    orc_metric m;
    metric_at(a, y[0], y[1], &m);
    double ur = y[3], ut = y[4], up = y[5];
    double uu = m.gi_rr * ur * ur + 2.0 * m.gi_rp * ur * up + m.gi_thth * ut * ut + m.gi_pp * up * up;
    double u0 = sqrt(eps + uu) / m.alpha;
    f[0] = (m.gi_rr * ur + m.gi_rp * up) / u0 - m.beta;
    f[1] = m.gi_thth * ut / u0;
    f[2] = (m.gi_rp * ur + m.gi_pp * up) / u0;
    for (int k = 0; k < 2; ++k) {
        double dguu = ur * ur * m.dgi_rr[k] + 2.0 * ur * up * m.dgi_rp[k] + ut * ut * m.dgi_thth[k] + up * up * m.dgi_pp[k];
        f[3 + k] = -m.alpha * u0 * m.da[k] + ur * m.db[k] - dguu / (2.0 * u0);
    }
    f[5] = 0.0;
}

void orc_geodesic_rhs(double a, double eps, const double *y, double *f) { geo_rhs(a, eps, y, f); }

static void lower(const orc_metric *m, const double v[3], double o[3])
{
    o[0] = m->g_rr * v[0] + m->g_rp * v[2];
    o[1] = m->g_thth * v[1];
    o[2] = m->g_rp * v[0] + m->g_pp * v[2];
}
static void raise_(const orc_metric *m, const double v[3], double o[3])
{
    o[0] = m->gi_rr * v[0] + m->gi_rp * v[2];
    o[1] = m->gi_thth * v[1];
    o[2] = m->gi_rp * v[0] + m->gi_pp * v[2];
}
/* covariant cross product (e_ijk v^j w^k), e_ijk = sqrt(gamma) eps_ijk */
static void cross(double sg, const double v[3], const double w[3], double o[3])
{
    o[0] = sg * (v[1] * w[2] - v[2] * w[1]);
    o[1] = sg * (v[2] * w[0] - v[0] * w[2]);
    o[2] = sg * (v[0] * w[1] - v[1] * w[0]);
}

/* Generalized Boris step over a full dt at fields n, Eqs. boris-plus-minus,
 * u0bar, boris-scheme. Dv, Bv contravariant D^j, B^k at the particle. */
static void boris(const orc_metric *m, double qm, double dt, const double Dv[3], const double Bv[3], double u[3])
{
    double Dl[3], um[3], uup[3], t[3], tl[3], s[3], cr[3], ut[3], up[3];
    lower(m, Dv, Dl);
    double h = qm * m->alpha * dt / 2.0;
    for (int k = 0; k < 3; ++k) um[k] = u[k] + h * Dl[k];
    raise_(m, um, uup);
    double uu = um[0] * uup[0] + um[1] * uup[1] + um[2] * uup[2];
    double u0b = sqrt(1.0 + uu) / m->alpha;
    for (int k = 0; k < 3; ++k) t[k] = qm * Bv[k] * dt / (2.0 * u0b);
    lower(m, t, tl);
    double tt = t[0] * tl[0] + t[1] * tl[1] + t[2] * tl[2];
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + tt);
    cross(m->sqrtg, uup, t, cr);
    for (int k = 0; k < 3; ++k) ut[k] = um[k] + cr[k];
    double utu[3];
    raise_(m, ut, utu);
    cross(m->sqrtg, utu, s, cr);
    for (int k = 0; k < 3; ++k) up[k] = um[k] + cr[k];
    for (int k = 0; k < 3; ++k) u[k] = up[k] + h * Dl[k];
}

void orc_boris(double a, double r, double th, double qm, double dt, const double *Dv, const double *Bv, double *u)
{
    orc_metric m;
    metric_at(a, r, th, &m);
    boris(&m, qm, dt, Dv, Bv, u);
}

/* The alternative momentum update of Sec. 2.2: transform to the FIDO frame
 * and apply Vay's update there (Vay 2008, Phys. Plasmas 15, 056701).
 *
 * FIDO frame: the orthonormal spatial triad e_(a) of the normal observer,
 *   e_(r)   = (1, 0, -g_rp/g_pp) / sqrt(g_rr - g_rp^2/g_pp),
 *   e_(th)  = (0, 1/sqrt(g_thth), 0),
 *   e_(ph)  = (0, 0, 1/sqrt(g_pp))            (contravariant components),
 * right-handed like (r, theta, phi).  A covector u_i has frame components
 * u_a = e^i_(a) u_i, a vector V^j has V_a = e^i_(a) gamma_ij V^j, and back
 * u_i = sum_a gamma_ij e^j_(a) u_a.  There the Lorentz force of Eq. Lorentz
 * is the flat one, with the FIDO's fields E = D and B and its proper time
 * d tau = alpha dt:  du/dtau = (q/m)(E + u x B / Gamma), Gamma = sqrt(1 + u.u).
 *
 * Vay's step over dtau, fields at n:
 *   u'     = u + (q/m) dtau (E + (u / Gamma) x B / 2)
 *   tau    = (q/m) dtau B / 2,   u* = u'.tau,   sigma = 1 + u'.u' - tau.tau
 *   Gamma1 = sqrt((sigma + sqrt(sigma^2 + 4 (tau.tau + u*^2))) / 2)
 *   t      = tau / Gamma1,        s = 1 / (1 + t.t)
 *   u1     = s (u' + (u'.t) t + u' x t).                                      */
static void vay_fido(const orc_metric *m, double qm, double dt, const double Dv[3], const double Bv[3], double u[3])
{
    double E[3][3] = {{0}};  /* E[a] = e^i_(a) (contravariant components) */
    double nr = sqrt(m->g_rr - m->g_rp * m->g_rp / m->g_pp);
    E[0][0] = 1.0 / nr;
    E[0][2] = -m->g_rp / m->g_pp / nr;
    E[1][1] = 1.0 / sqrt(m->g_thth);
    E[2][2] = 1.0 / sqrt(m->g_pp);
    double Dl[3], Bl[3];
    lower(m, Dv, Dl);
    lower(m, Bv, Bl);
    double uf[3], Ef[3], Bf[3];
    for (int a = 0; a < 3; ++a) {
        uf[a] = Ef[a] = Bf[a] = 0.0;
        for (int i = 0; i < 3; ++i) {
            uf[a] += E[a][i] * u[i];
            Ef[a] += E[a][i] * Dl[i];
            Bf[a] += E[a][i] * Bl[i];
        }
    }
    double dtau = m->alpha * dt;
    double G = sqrt(1.0 + uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
    double vxB[3] = {(uf[1] * Bf[2] - uf[2] * Bf[1]) / G, (uf[2] * Bf[0] - uf[0] * Bf[2]) / G,
                     (uf[0] * Bf[1] - uf[1] * Bf[0]) / G};
    double up[3], tau[3];
    for (int a = 0; a < 3; ++a) {
        up[a] = uf[a] + qm * dtau * (Ef[a] + 0.5 * vxB[a]);
        tau[a] = 0.5 * qm * dtau * Bf[a];
    }
    double us = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
    double tt = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    double sigma = 1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2] - tt;
    double G1 = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tt + us * us))));
    double t[3] = {tau[0] / G1, tau[1] / G1, tau[2] / G1};
    double s = 1.0 / (1.0 + (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]));
    double ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
    double u1[3] = {s * (up[0] + ut * t[0] + (up[1] * t[2] - up[2] * t[1])),
                    s * (up[1] + ut * t[1] + (up[2] * t[0] - up[0] * t[2])),
                    s * (up[2] + ut * t[2] + (up[0] * t[1] - up[1] * t[0]))};
    /* back to the coordinate covector: u_i = gamma_ij e^j_(a) u1_a */
    double w[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) w[j] += E[a][j] * u1[a];
    lower(m, w, u);
}

void orc_vay(double a, double r, double th, double qm, double dt, const double *Dv, const double *Bv, double *u)
{
    orc_metric m;
    metric_at(a, r, th, &m);
    vay_fido(&m, qm, dt, Dv, Bv, u);
}

/* Momentum update (generalized Boris, or Vay in the FIDO frame; skipped for
 * photons or q = 0) then the geodesic predictor (Eq. geodesic-predictor) and
 * n_iter trapezoidal correctors (Eq. geodesic-corrector), each re-evaluated
 * at the latest iterate. y[2] = phi. */
static void push_core(double a, double qm, int massive, double dt, int n_iter,
                      const double Dv[3], const double Bv[3], double y[6], int pusher)
{
    if (massive && qm != 0.0) {
        orc_metric m;
        metric_at(a, y[0], y[1], &m);
        if (pusher == 1)
            vay_fido(&m, qm, dt, Dv, Bv, &y[3]);
        else
            boris(&m, qm, dt, Dv, Bv, &y[3]);
    }
    double eps = massive ? 1.0 : 0.0;
    double y0[6], f0[6], yt[6], ft[6];
    memcpy(y0, y, sizeof y0);
    geo_rhs(a, eps, y0, f0);
    for (int k = 0; k < 6; ++k) yt[k] = y0[k] + f0[k] * dt;
    for (int it = 0; it < n_iter; ++it) {
        geo_rhs(a, eps, yt, ft);
        for (int k = 0; k < 6; ++k) yt[k] = y0[k] + 0.5 * dt * (ft[k] + f0[k]);
    }
    memcpy(y, yt, sizeof yt);
}

/* one push with given field values (for pins of the pusher) */
void orc_push_values(double a, double qm, int massive, double dt, int n_iter, const double *Dv, const double *Bv, double *y)
{
    push_core(a, qm, massive, dt, n_iter, Dv, Bv, y, 0);
}

/* nsteps pushes with fields from the closed-form solution evaluated at x^n
 * (no grid); y is advanced in place and every `every` steps the state is
 * appended to traj (6 doubles per sample). Returns the number of samples. */
int orc_push_analytic(int kind, double B0, double a, double qm, int massive, double dt, int n_iter,
                      double *y, long nsteps, long every, double *traj)
{
    int ns = 0;
    for (long s = 0; s < nsteps; ++s) {
        double Dv[3] = {0, 0, 0}, Bv[3] = {0, 0, 0};
        if (B0 != 0.0) closed_D(kind, a, B0, y[0], y[1], Dv, Bv);
        push_core(a, qm, massive, dt, n_iter, Dv, Bv, y, 0);
        if (every > 0 && (s + 1) % every == 0) {
            memcpy(traj + 6 * ns, y, 6 * sizeof(double));
            ++ns;
        }
    }
    return ns;
}

/* ------------------------------------------------------------------------ */
/* Field interpolation to the particle: bilinear CIC in logical coordinates */
/* on each component's own staggered lattice.  Rows beyond the axis mirror  */
/* the first interior row; theta components change sign there, r and phi   */
/* components do not (the map (theta, phi) -> (-theta, phi + pi)).          */
/* ------------------------------------------------------------------------ */
static double row_val(const orc_cfg *c, const double *F, int i, int j, double par)
{
    if (j < 0) return par * F[IDX(c, i, -1 - j)];
    if (j > c->nth) return par * F[IDX(c, i, 2 * c->nth - j)];
    return F[IDX(c, i, j)];
}
static double row_val_half(const orc_cfg *c, const double *F, int i, int j, double par)
{
    /* half-theta lattice: row j is theta_{j+1/2}; row -1 mirrors row 0 and
     * row nth mirrors row nth-1 */
    if (j < 0) return par * F[IDX(c, i, -1 - j)];
    if (j > c->nth - 1) return par * F[IDX(c, i, 2 * c->nth - 1 - j)];
    return F[IDX(c, i, j)];
}

static double interp(const orc_cfg *c, const double *F, double x1, double x2, double sr, int half_t, double par)
{
    double xi = x1 - sr, eta = x2 - (half_t ? 0.5 : 0.0);
    int i = (int)floor(xi);
    int j = (int)floor(eta);
    if (!half_t && j > c->nth - 1) j = c->nth - 1;
    double f = xi - i, gg = eta - j;
    double v00, v10, v01, v11;
    if (half_t) {
        v00 = row_val_half(c, F, i, j, par); v10 = row_val_half(c, F, i + 1, j, par);
        v01 = row_val_half(c, F, i, j + 1, par); v11 = row_val_half(c, F, i + 1, j + 1, par);
    } else {
        v00 = row_val(c, F, i, j, par); v10 = row_val(c, F, i + 1, j, par);
        v01 = row_val(c, F, i, j + 1, par); v11 = row_val(c, F, i + 1, j + 1, par);
    }
    return (1 - f) * (1 - gg) * v00 + f * (1 - gg) * v10 + (1 - f) * gg * v01 + f * gg * v11;
}

static void interp_fields(const orc_cfg *c, double *const D[3], double *const B[3], double x1, double x2,
                          double Dv[3], double Bv[3])
{
    Dv[0] = interp(c, D[0], x1, x2, 0.5, 0, 1.0);
    Dv[1] = interp(c, D[1], x1, x2, 0.0, 1, -1.0);
    Dv[2] = interp(c, D[2], x1, x2, 0.0, 0, 1.0);
    Bv[0] = interp(c, B[0], x1, x2, 0.0, 1, 1.0);
    Bv[1] = interp(c, B[1], x1, x2, 0.5, 0, 1.0);
    Bv[2] = interp(c, B[2], x1, x2, 0.5, 1, 1.0);
}

/* ------------------------------------------------------------------------ */
/* Third-order spline shape (Sec. 2.3's configuration option): the cubic    */
/* B-spline in logical units, the convolution of four unit boxes,           */
/*   W3(x) = 2/3 - x^2 + |x|^3/2        for |x| < 1,                         */
/*         = (2 - |x|)^3 / 6            for 1 <= |x| < 2,   0 beyond,        */
/* and S = W3(x1 - i) W3(x2 - j) on each lattice.  Rows past the polar axis */
/* are the mirror rows of the relabelling (r, -theta, phi + pi) of the same */
/* point: theta components change sign, r and phi components do not.       */
/* ------------------------------------------------------------------------ */
static double W3(double d)
{
    d = fabs(d);
    if (d < 1.0) return 2.0 / 3.0 - d * d + 0.5 * d * d * d;
    if (d < 2.0) { double e = 2.0 - d; return e * e * e / 6.0; }
    return 0.0;
}

/* mirror of row j and its parity: integer (vertex) rows theta_j = j dth,
 * half rows theta_{j+1/2} */
double orc_w3(double d) { return W3(d); }

static int mirror_row(const orc_cfg *c, int j, int half_t, int *flip)
{
    *flip = 0;
    int top = half_t ? c->nth - 1 : c->nth;
    if (j < 0) { *flip = 1; return half_t ? -1 - j : -j; }
    if (j > top) { *flip = 1; return half_t ? 2 * c->nth - 1 - j : 2 * c->nth - j; }
    return j;
}

static double interp3(const orc_cfg *c, const double *F, double x1, double x2, double sr, int half_t, double par)
{
    double xi = x1 - sr, eta = x2 - (half_t ? 0.5 : 0.0);
    int i = (int)floor(xi), j = (int)floor(eta);
    double v = 0.0;
    for (int a = -1; a <= 2; ++a) {
        double wr = W3(xi - (i + a));
        for (int b = -1; b <= 2; ++b) {
            int flip, jj = mirror_row(c, j + b, half_t, &flip);
            v += wr * W3(eta - (j + b)) * (flip ? par : 1.0) * F[IDX(c, i + a, jj)];
        }
    }
    return v;
}

static void interp_fields3(const orc_cfg *c, double *const D[3], double *const B[3], double x1, double x2,
                           double Dv[3], double Bv[3])
{
    Dv[0] = interp3(c, D[0], x1, x2, 0.5, 0, 1.0);
    Dv[1] = interp3(c, D[1], x1, x2, 0.0, 1, -1.0);
    Dv[2] = interp3(c, D[2], x1, x2, 0.0, 0, 1.0);
    Bv[0] = interp3(c, B[0], x1, x2, 0.0, 1, 1.0);
    Bv[1] = interp3(c, B[1], x1, x2, 0.5, 0, -1.0);
    Bv[2] = interp3(c, B[2], x1, x2, 0.5, 1, 1.0);
}

void orc_interp(const orc_cfg *c, double *D0, double *D1, double *D2, double *B0r, double *B1, double *B2,
                double x1, double x2, double *out6)
{
    double *D[3] = {D0, D1, D2}, *B[3] = {B0r, B1, B2};
    if (c->shape == 3)
        interp_fields3(c, D, B, x1, x2, out6, out6 + 3);
    else
        interp_fields(c, D, B, x1, x2, out6, out6 + 3);
}

/* Eq. esirkepov-decomp and j-phi-deposit with the cubic shape: the window
 * spans the 5 x 5 vertices (b1 .. b1+4, b2 .. b2+4) around both positions
 * (b = the lower of the two cells, minus 1); W_r, W_theta from the four shape
 * products, prefix sums along r (J^r A at faces b1+A+1/2) and theta.  Entries
 * past the polar axis are added to their mirror entries (J^r A, J^phi even,
 * J^theta A odd; the axis rows are their own mirrors); columns past the
 * storage (a particle leaving through r_out) are dropped. */
static void fold_add(const orc_cfg *c, double *F, int i, int j, int half_t, double odd, double v)
{
    if (v == 0.0 || i < -c->ng || i > c->nr + c->ng - 1) return;
    int flip, jj = mirror_row(c, j, half_t, &flip);
    F[IDX(c, i, jj)] += flip ? odd * v : v;
}

static void deposit_one3(const orc_cfg *c, const double *dV, double *JrA, double *JtA, double *Jph,
                         double qw, double r0x, double t0x, double r1x, double t1x, double dphi)
{
    int fr0 = (int)floor(r0x), fr1 = (int)floor(r1x);
    int b1 = (fr0 < fr1 ? fr0 : fr1) - 1;
    int j0 = (int)floor(t0x), j1 = (int)floor(t1x);
    int b2 = (j0 < j1 ? j0 : j1) - 1;
    double Wr[5][5], Wt[5][5];
    for (int A = 0; A < 5; ++A)
        for (int Bb = 0; Bb < 5; ++Bb) {
            int k = b1 + A, l = b2 + Bb;
            double S00 = W3(r0x - k) * W3(t0x - l);
            double S11 = W3(r1x - k) * W3(t1x - l);
            double S10 = W3(r1x - k) * W3(t0x - l);
            double S01 = W3(r0x - k) * W3(t1x - l);
            Wr[A][Bb] = S11 - S01 + S10 - S00;
            Wt[A][Bb] = S11 - S10 + S01 - S00;
            double sbar = S11 / 3.0 + S10 / 6.0 + S01 / 6.0 + S00 / 3.0;
            if (sbar != 0.0) {
                int flip, ll = mirror_row(c, l, 0, &flip);
                if (k >= -c->ng && k <= c->nr + c->ng - 1)
                    Jph[IDX(c, k, ll)] += qw * (dphi / c->dt) * sbar / dV[IDX(c, k, ll)];
            }
        }
    for (int Bb = 0; Bb < 5; ++Bb) {
        double acc = 0.0;
        for (int A = 0; A < 4; ++A) {
            acc += Wr[A][Bb];
            fold_add(c, JrA, b1 + A, b2 + Bb, 0, 1.0, -qw / (2.0 * c->dt) * acc);
        }
    }
    for (int A = 0; A < 5; ++A) {
        double acc = 0.0;
        for (int Bb = 0; Bb < 4; ++Bb) {
            acc += Wt[A][Bb];
            fold_add(c, JtA, b1 + A, b2 + Bb, 1, -1.0, -qw / (2.0 * c->dt) * acc);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Charge-conserving deposit, Sec. 2.3: Esirkepov decomposition of Eq.      */
/* esirkepov-decomp with CIC S_ij, local prefix sums for J^r A_r and         */
/* J^th A_th (from Eq. J-integral-eqn), J^phi by Eq. j-phi-deposit.          */
/* ------------------------------------------------------------------------ */
static double W1(double d)
{
    d = fabs(d);
    return d < 1.0 ? 1.0 - d : 0.0;
}

static int jcell(const orc_cfg *c, double x2)
{
    int j = (int)floor(x2);
    if (j > c->nth - 1) j = c->nth - 1;
    return j;
}

/* JrA at D^r locations, JtA at D^th locations, Jph at vertices (divided by
 * dV = A^D_phi, dphi = 1). */
static void deposit_one(const orc_cfg *c, const double *dV, double *JrA, double *JtA, double *Jph,
                        double qw, double r0x, double t0x, double r1x, double t1x, double dphi)
{
    int b1 = (int)floor(r0x) < (int)floor(r1x) ? (int)floor(r0x) : (int)floor(r1x);
    int j0 = jcell(c, t0x), j1 = jcell(c, t1x);
    int b2 = j0 < j1 ? j0 : j1;
    if (b2 > c->nth - 2) b2 = c->nth - 2;
    double Wr[3][3], Wt[3][3];
    for (int A = 0; A < 3; ++A)
        for (int Bb = 0; Bb < 3; ++Bb) {
            int k = b1 + A, l = b2 + Bb;
            double S00 = W1(r0x - k) * W1(t0x - l);
            double S11 = W1(r1x - k) * W1(t1x - l);
            double S10 = W1(r1x - k) * W1(t0x - l); /* r at n+1, theta at n */
            double S01 = W1(r0x - k) * W1(t1x - l); /* r at n, theta at n+1 */
            Wr[A][Bb] = S11 - S01 + S10 - S00;
            Wt[A][Bb] = S11 - S10 + S01 - S00;
            double sbar = S11 / 3.0 + S10 / 6.0 + S01 / 6.0 + S00 / 3.0;
            if (sbar != 0.0) Jph[IDX(c, k, l)] += qw * (dphi / c->dt) * sbar / dV[IDX(c, k, l)];
        }
    for (int Bb = 0; Bb < 3; ++Bb) {
        double acc = 0.0;
        for (int A = 0; A < 2; ++A) {
            acc += Wr[A][Bb];
            JrA[IDX(c, b1 + A, b2 + Bb)] += -qw / (2.0 * c->dt) * acc;
        }
    }
    for (int A = 0; A < 3; ++A) {
        double acc = 0.0;
        for (int Bb = 0; Bb < 2; ++Bb) {
            acc += Wt[A][Bb];
            JtA[IDX(c, b1 + A, b2 + Bb)] += -qw / (2.0 * c->dt) * acc;
        }
    }
}

/* single-particle deposit into caller arrays (for pins P10, P12) */
void orc_deposit_one(const orc_cfg *c, double *JrA, double *JtA, double *Jph, double qw,
                     double r0x, double t0x, double r1x, double t1x, double dphi)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    if (c->shape == 3)
        deposit_one3(c, g.AD[2], JrA, JtA, Jph, qw, r0x, t0x, r1x, t1x, dphi);
    else
        deposit_one(c, g.AD[2], JrA, JtA, Jph, qw, r0x, t0x, r1x, t1x, dphi);
}

/* ------------------------------------------------------------------------ */
/* Push + deposit over all particles (Fig. stepping): Boris at x^n with     */
/* fields n, geodesic to x^{n+1}, axis reflection, Esirkepov deposit from   */
/* x^n to x^{n+1}; then J = (J A)/A^D.  Particles that leave [r_in, r_out)  */
/* are flagged dead after their deposit; moves of more than one cell or     */
/* non-finite states flag the particle dead and set a status.               */
/* ------------------------------------------------------------------------ */
/* one particle: returns its status (ORC_OK, ORC_ENAN or ORC_ERANGE) */
static int push_deposit_one(const orc_cfg *c, const orc_geom *g, double lnrin, long p, double *pr, double *pth,
                            double *pu1, double *pu2, double *pu3, uint32_t *tag, double *dphi_out,
                            double *const D[3], double *const B[3], double *J0, double *J1, double *J2)
{
    if (tag[p] & ORC_DEAD) { if (dphi_out) dphi_out[p] = 0.0; return ORC_OK; }
    int sp = tag[p] & 3u;
    double y[6] = {pr[p], pth[p], 0.0, pu1[p], pu2[p], pu3[p]};
    double x1a = (log(y[0]) - lnrin) / c->dx1, x2a = y[1] / c->dth;
    double Dv[3], Bv[3];
    if (c->shape == 3)
        interp_fields3(c, D, B, x1a, x2a, Dv, Bv);
    else
        interp_fields(c, D, B, x1a, x2a, Dv, Bv);
    push_core(c->a, c->qm[sp], c->massive[sp], c->dt, c->n_push_iter, Dv, Bv, y, c->pusher);
    /* axis reflection */
    if (y[1] < 0.0) { y[1] = -y[1]; y[4] = -y[4]; }
    if (y[1] > M_PI) { y[1] = 2.0 * M_PI - y[1]; y[4] = -y[4]; }
    int bad = 0;
    for (int k = 0; k < 6; ++k) if (!isfinite(y[k])) bad = 1;
    if (bad) { tag[p] |= ORC_DEAD; if (dphi_out) dphi_out[p] = 0.0; return ORC_ENAN; }
    double x1b = (log(y[0]) - lnrin) / c->dx1, x2b = y[1] / c->dth;
    int di = (int)floor(x1b) - (int)floor(x1a);
    int dj = jcell(c, x2b) - jcell(c, x2a);
    if (di < -1 || di > 1 || dj < -1 || dj > 1) {
        tag[p] |= ORC_DEAD;
        if (dphi_out) dphi_out[p] = 0.0;
        return ORC_ERANGE;
    }
    if (c->shape == 3)
        deposit_one3(c, g->AD[2], J0, J1, J2, c->qw[sp], x1a, x2a, x1b, x2b, y[2]);
    else
        deposit_one(c, g->AD[2], J0, J1, J2, c->qw[sp], x1a, x2a, x1b, x2b, y[2]);
    pr[p] = y[0]; pth[p] = y[1]; pu1[p] = y[3]; pu2[p] = y[4]; pu3[p] = y[5];
    if (dphi_out) dphi_out[p] = y[2];
    if (y[0] < c->r_in || y[0] >= c->r_out) tag[p] |= ORC_DEAD;
    return ORC_OK;
}

int orc_push_deposit(const orc_cfg *c, long np, double *pr, double *pth, double *pu1, double *pu2, double *pu3,
                     uint32_t *tag, double *dphi_out,
                     double *D0, double *D1, double *D2, double *B0r, double *B1, double *B2,
                     double *J0, double *J1, double *J2)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    double *D[3] = {D0, D1, D2}, *B[3] = {B0r, B1, B2};
    memset(J0, 0, g.n * sizeof(double));
    memset(J1, 0, g.n * sizeof(double));
    memset(J2, 0, g.n * sizeof(double));
    int status = ORC_OK;
    double lnrin = log(c->r_in);
    int nt = orc_nthreads;
    if (nt <= 1) {
        for (long p = 0; p < np; ++p) {
            int st = push_deposit_one(c, &g, lnrin, p, pr, pth, pu1, pu2, pu3, tag, dphi_out, D, B, J0, J1, J2);
            if (st && !status) status = st;
        }
    } else {
        /* thread t pushes particles [t np / nt, (t+1) np / nt) into its own
         * current arrays; the first status in particle order is kept */
        double *Jt = calloc((size_t)nt * 3 * g.n, sizeof(double));
        int *stt = calloc(nt, sizeof(int));
#pragma omp parallel for schedule(static, 1) num_threads(nt)
        for (int t = 0; t < nt; ++t) {
            double *j0 = Jt + (size_t)t * 3 * g.n, *j1 = j0 + g.n, *j2 = j1 + g.n;
            for (long p = (long)t * np / nt; p < (long)(t + 1) * np / nt; ++p) {
                int st = push_deposit_one(c, &g, lnrin, p, pr, pth, pu1, pu2, pu3, tag, dphi_out, D, B, j0, j1, j2);
                if (st && !stt[t]) stt[t] = st;
            }
        }
        for (int t = 0; t < nt; ++t) {
            const double *j0 = Jt + (size_t)t * 3 * g.n, *j1 = j0 + g.n, *j2 = j1 + g.n;
            for (int q = 0; q < g.n; ++q) { J0[q] += j0[q]; J1[q] += j1[q]; J2[q] += j2[q]; }
            if (stt[t] && !status) status = stt[t];
        }
        free(Jt);
        free(stt);
    }
    /* "after finishing the current deposition loop, we divide the results by
     * A^D_r and A^D_theta" (Sec. 2.3) */
    for (int q = 0; q < g.n; ++q) {
        if (g.AD[0][q] != 0.0) J0[q] /= g.AD[0][q];
        if (g.AD[1][q] != 0.0) J1[q] /= g.AD[1][q];
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Stable counting sort by cell key (cell = j*nr + i; dead -> nr*nth), with */
/* the dead particles dropped.  perm[k] = old index of new slot k.          */
/* Returns the number of live particles.                                    */
/* ------------------------------------------------------------------------ */
static long cell_key(const orc_cfg *c, double r, double th, uint32_t tag)
{
    long ncell = (long)c->nr * c->nth;
    if (tag & ORC_DEAD) return ncell;
    double x1 = (log(r) - log(c->r_in)) / c->dx1;
    int i = (int)floor(x1);
    int j = jcell(c, th / c->dth);
    if (i < 0 || i >= c->nr || j < 0) return ncell;
    return (long)j * c->nr + i;
}

void orc_cell_keys(const orc_cfg *c, long np, const double *pr, const double *pth, const uint32_t *tag, int32_t *key)
{
    for (long p = 0; p < np; ++p) key[p] = (int32_t)cell_key(c, pr[p], pth[p], tag[p]);
}

long orc_counting_sort(long np, long nkeys, const int32_t *key, int64_t *perm)
{
    long *count = calloc(nkeys + 1, sizeof(long));
    for (long p = 0; p < np; ++p) count[key[p]]++;
    long run = 0;
    for (long k = 0; k <= nkeys; ++k) { long t = count[k]; count[k] = run; run += t; }
    for (long p = 0; p < np; ++p) perm[count[key[p]]++] = p;
    long live = 0;
    /* live = number with key < nkeys (dead key == nkeys sorts last) */
    for (long p = 0; p < np; ++p) if (key[p] < nkeys) ++live;
    free(count);
    return live;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics: charge density rho = sum q w S / dV at vertices; discrete   */
/* div D (Eq. D-B-evolution, first line, in the integral form of Eq.         */
/* J-integral-eqn); div B flux sum per primal cell.                          */
/* ------------------------------------------------------------------------ */
void orc_rho(const orc_cfg *c, long np, const double *pr, const double *pth, const uint32_t *tag, double *rho)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    memset(rho, 0, g.n * sizeof(double));
    double lnrin = log(c->r_in);
    for (long p = 0; p < np; ++p) {
        if (tag[p] & ORC_DEAD) continue;
        double x1 = (log(pr[p]) - lnrin) / c->dx1, x2 = pth[p] / c->dth;
        if (c->shape == 3) {
            int i = (int)floor(x1), j = (int)floor(x2);
            for (int A = -1; A <= 2; ++A)
                for (int Bb = -1; Bb <= 2; ++Bb) {
                    int k = i + A, l = j + Bb, flip;
                    if (k < -c->ng || k > c->nr + c->ng - 1) continue;
                    int ll = mirror_row(c, l, 0, &flip);
                    double S = W3(x1 - k) * W3(x2 - l);
                    rho[IDX(c, k, ll)] += c->qw[tag[p] & 3u] * S / g.AD[2][IDX(c, k, ll)];
                }
            continue;
        }
        int i = (int)floor(x1), j = jcell(c, x2);
        for (int A = 0; A < 2; ++A)
            for (int Bb = 0; Bb < 2; ++Bb) {
                int k = i + A, l = j + Bb;
                double S = W1(x1 - k) * W1(x2 - l);
                rho[IDX(c, k, l)] += c->qw[tag[p] & 3u] * S / g.AD[2][IDX(c, k, l)];
            }
    }
}

void orc_divD(const orc_cfg *c, const double *D0, const double *D1, double *divD)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    memset(divD, 0, g.n * sizeof(double));
    for (int j = 0; j <= c->nth; ++j)
        for (int i = -c->ng + 1; i < c->ld - c->ng; ++i) {
            int q = IDX(c, i, j), qm = IDX(c, i - 1, j);
            double flux = D0[q] * g.AD[0][q] - D0[qm] * g.AD[0][qm];
            if (j < c->nth) flux += D1[q] * g.AD[1][q];
            if (j > 0) flux -= D1[IDX(c, i, j - 1)] * g.AD[1][IDX(c, i, j - 1)];
            divD[q] = flux / g.AD[2][q];
        }
}

void orc_divB(const orc_cfg *c, const double *B0r, const double *B1, double *divB)
{
    orc_geom g = *geom_get(c); /* shallow copy of the cached tables */
    memset(divB, 0, g.n * sizeof(double));
    for (int j = 0; j < c->nth; ++j)
        for (int i = -c->ng; i < c->ld - c->ng - 1; ++i) {
            int q = IDX(c, i, j), qp = IDX(c, i + 1, j), qj = IDX(c, i, j + 1);
            divB[q] = B0r[qp] * g.AB[0][qp] - B0r[q] * g.AB[0][q] + B1[qj] * g.AB[1][qj] - B1[q] * g.AB[1][q];
        }
}

/* ======================================================================== */
/* Batched 1D spark gaps (the radiative pair-production prescription of     */
/* Sec. 4, Eq. optical-depth, on single radial field lines).                 */
/*                                                                          */
/* The paper runs its spark gaps in 2D; this 1D line model is the reading   */
/* used here: along a monopole field line at                              */
/* fixed theta_k particles slide radially (theta frozen, u_theta = 0, u_phi */
/* kept), the electric kick is the covariant gamma_rr D^r part of the Boris */
/* step, the geodesic step is Eq. geodesic-predictor/-corrector restricted  */
/* to (r, u_r), the deposit is the 1D Esirkepov prefix sum, and the one     */
/* field component obeys d(A_r D^r)/dt = I_0 - J^r A_r with an imposed line */
/* current I_0 (constant along the line, so charge is conserved).           */
/* Radiation (Sec. 4): a charged particle whose FIDO Lorentz factor         */
/* Gamma = alpha u^0 reaches gamma_thr emits a photon of FIDO energy eps_ph */
/* along its momentum and loses that energy; photons follow geodesics with  */
/* epsilon = 0 and convert with probability 1 - exp(-tau dt) per step into  */
/* an e-/e+ pair sharing the photon's FIDO energy equally, along its        */
/* direction (conversion requires energy > 2).                              */
/* ======================================================================== */

/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of two     */
/* 64x64->128 multiplications with the Weyl-sequence key schedule.          */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out)
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t h0, l0, h1, l1;
        mulhilo64(0xD2E7470EE14C6C93ULL, x0, &h0, &l0);
        mulhilo64(0xCA5A826395121157ULL, x2, &h1, &l1);
        uint64_t y0 = h1 ^ x1 ^ k0, y1 = l1, y2 = h0 ^ x3 ^ k1, y3 = l0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* splitmix64 finaliser (Steele, Lea & Flood 2014) */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* identity of the k-th particle created by `parent` at step `step` */
uint64_t orc_child_id(uint64_t parent, int64_t step, int k)
{
    return orc_splitmix64(orc_splitmix64(parent) ^ (((uint64_t)step << 2) | (uint64_t)k));
}

/* uniform in [0,1) with 53 random bits from counter (id, step, event, 0) */
double orc_uniform(uint64_t seed, uint64_t id, int64_t step, int event)
{
    uint64_t ctr[4] = {id, (uint64_t)step, (uint64_t)event, 0}, key[2] = {seed, 0}, out[4];
    orc_philox4x64(ctr, key, out);
    return (double)(out[0] >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct {
    int n;                       /* cells along the line                     */
    double a, theta, r_in, r_out, dx1;
    double dt;
    int n_push_iter;
    double qm[4], qw[4];
    int massive[4];
    double I0;                   /* imposed line current (J A units)        */
    double gamma_thr, eps_ph, tau;
    uint64_t seed;
} orc_line;

static double line_r(const orc_line *L, double x) { return L->r_in * exp(x * L->dx1); }

/* A_r of the flux tube at D^r location i+1/2 (per unit theta and phi) */
void orc_line_area(const orc_line *L, double *A)
{
    for (int i = 0; i < L->n; ++i) {
        orc_metric m;
        metric_at(L->a, line_r(L, i + 0.5), L->theta, &m);
        A[i] = m.sqrtg;
    }
}

/* D^r on the line from the monopole closed form (App. C) */
void orc_line_init_D(const orc_line *L, double B0, double *D)
{
    for (int i = 0; i < L->n; ++i) {
        double Dv[3], Bu[3];
        closed_D(2, L->a, B0, line_r(L, i + 0.5), L->theta, Dv, Bu);
        D[i] = Dv[0];
    }
}

static double line_D_at(const orc_line *L, const double *D, double x)
{
    double xi = x - 0.5;
    int i = (int)floor(xi);
    double f = xi - i;
    int i0 = i < 0 ? 0 : (i > L->n - 1 ? L->n - 1 : i);
    int i1 = i + 1 < 0 ? 0 : (i + 1 > L->n - 1 ? L->n - 1 : i + 1);
    return (1.0 - f) * D[i0] + f * D[i1];
}

static double line_gamma(const orc_line *L, double r, double ur, double up, double eps)
{
    orc_metric m;
    metric_at(L->a, r, L->theta, &m);
    return sqrt(eps + m.gi_rr * ur * ur + 2.0 * m.gi_rp * ur * up + m.gi_pp * up * up);
}

/* One step of one line.  Arrays hold *np particles (capacity cap): logical
 * position x1, covariant u_r, u_phi, tag (species | DEAD), id.  D has n
 * entries, JA (output) n+2 faces (index f+1 for face f = -1..n).  Survivors
 * keep their order; particles created this step follow in parent order.
 * counts[0] = photons emitted, counts[1] = photons converted. */
int orc_line_step(const orc_line *L, int64_t step, long *np, long cap, double *x1, double *ur, double *up,
                  uint32_t *tag, uint64_t *id, double *D, double *JA, long *counts)
{
    int status = ORC_OK;
    long n0 = *np, nnew = 0;
    double *nx = malloc(sizeof(double) * (2 * n0 + 2));
    double *nur = malloc(sizeof(double) * (2 * n0 + 2));
    double *nup = malloc(sizeof(double) * (2 * n0 + 2));
    uint32_t *ntag = malloc(sizeof(uint32_t) * (2 * n0 + 2));
    uint64_t *nid = malloc(sizeof(uint64_t) * (2 * n0 + 2));
    double *A = malloc(sizeof(double) * L->n);
    orc_line_area(L, A);
    memset(JA, 0, sizeof(double) * (L->n + 2));
    counts[0] = counts[1] = 0;
    double Pconv = 1.0 - exp(-L->tau * L->dt);
    for (long p = 0; p < n0; ++p) {
        if (tag[p] & ORC_DEAD) continue;
        int sp = tag[p] & 3u;
        int massive = L->massive[sp];
        double xa = x1[p];
        double y[6] = {line_r(L, xa), L->theta, 0.0, ur[p], 0.0, up[p]};
        if (massive && L->qm[sp] != 0.0) {
            /* electric part of the Boris step along the line: u_r += (q/m) alpha dt gamma_rr D^r */
            orc_metric m;
            metric_at(L->a, y[0], L->theta, &m);
            y[3] += L->qm[sp] * m.alpha * L->dt * m.g_rr * line_D_at(L, D, xa);
        }
        /* geodesic predictor-corrector restricted to (r, u_r) */
        double eps = massive ? 1.0 : 0.0;
        double y0[6], f0[6], yt[6], ft[6];
        memcpy(y0, y, sizeof y0);
        geo_rhs(L->a, eps, y0, f0);
        memcpy(yt, y0, sizeof yt);
        yt[0] = y0[0] + L->dt * f0[0];
        yt[3] = y0[3] + L->dt * f0[3];
        for (int it = 0; it < L->n_push_iter; ++it) {
            geo_rhs(L->a, eps, yt, ft);
            yt[0] = y0[0] + 0.5 * L->dt * (ft[0] + f0[0]);
            yt[3] = y0[3] + 0.5 * L->dt * (ft[3] + f0[3]);
        }
        if (!isfinite(yt[0]) || !isfinite(yt[3]) || yt[0] <= 0.0) {
            tag[p] |= ORC_DEAD;
            status = status ? status : ORC_ENAN;
            continue;
        }
        double xb = log(yt[0] / L->r_in) / L->dx1;
        int i0 = (int)floor(xa), di = (int)floor(xb) - i0;
        if (di < -1 || di > 1) {
            tag[p] |= ORC_DEAD;
            status = status ? status : ORC_ERANGE;
            continue;
        }
        if (L->qw[sp] != 0.0) {
            /* 1D Esirkepov: J A(face k+1/2) = -(q/dt) sum_{k'<=k} (S1 - S0)(k') */
            double acc = 0.0;
            for (int k = i0 - 1; k <= i0 + 2; ++k) {
                acc += W1(xb - k) - W1(xa - k);
                if (k >= -1 && k <= L->n) JA[k + 1] += -L->qw[sp] / L->dt * acc;
            }
        }
        x1[p] = xb;
        ur[p] = yt[3];
        double r = yt[0];
        if (r < L->r_in || r >= L->r_out) { tag[p] |= ORC_DEAD; continue; }
        if (massive && L->qm[sp] != 0.0) {
            double G = line_gamma(L, r, ur[p], up[p], 1.0);
            if (G >= L->gamma_thr) {
                double pm = sqrt(G * G - 1.0), G2 = G - L->eps_ph, pm2 = sqrt(G2 * G2 - 1.0);
                double kr = L->eps_ph * ur[p] / pm, kp = L->eps_ph * up[p] / pm;
                ur[p] *= pm2 / pm;
                up[p] *= pm2 / pm;
                nx[nnew] = xb; nur[nnew] = kr; nup[nnew] = kp; ntag[nnew] = 3u;
                nid[nnew] = orc_child_id(id[p], step, 0);
                ++nnew;
                counts[0]++;
            }
        } else if (!massive) {
            double e = line_gamma(L, r, ur[p], up[p], 0.0);
            double u = orc_uniform(L->seed, id[p], step, 1);
            if (e > 2.0 && u < Pconv) {
                double pp = sqrt(0.25 * e * e - 1.0), s = pp / e;
                tag[p] |= ORC_DEAD;
                for (int k = 0; k < 2; ++k) {
                    nx[nnew] = xb; nur[nnew] = s * ur[p]; nup[nnew] = s * up[p]; ntag[nnew] = (uint32_t)k;
                    nid[nnew] = orc_child_id(id[p], step, 1 + k);
                    ++nnew;
                }
                counts[1]++;
            }
        }
    }
    /* field: d(A D)/dt = I0 - J A at every D^r location */
    for (int i = 0; i < L->n; ++i) D[i] += L->dt * (L->I0 - JA[i + 1]) / A[i];
    /* compaction: survivors in order, then the new particles in parent order */
    long w = 0;
    for (long p = 0; p < n0; ++p) {
        if (tag[p] & ORC_DEAD) continue;
        x1[w] = x1[p]; ur[w] = ur[p]; up[w] = up[p]; tag[w] = tag[p]; id[w] = id[p];
        ++w;
    }
    for (long k = 0; k < nnew; ++k) {
        if (w >= cap) { status = status ? status : 6; break; }
        x1[w] = nx[k]; ur[w] = nur[k]; up[w] = nup[k]; tag[w] = ntag[k]; id[w] = nid[k];
        ++w;
    }
    *np = w;
    free(nx); free(nur); free(nup); free(ntag); free(nid); free(A);
    return status;
}

/* ======================================================================== */
/* Objective of the differentiable form: the radial Poynting flux through   */
/* the vertex ring i_H nearest the horizon, sum over theta cells of         */
/* (E_theta H_phi - E_phi H_theta) dtheta (dphi = 1), with E_i, H_i the      */
/* auxiliary fields of Eq. E-H-B-D (App. B forms) and every factor brought  */
/* to (i_H, j+1/2) by the two- or four-point averages of the Yee layout.    */
/* ======================================================================== */
double orc_horizon_flux(const orc_cfg *c, double *D0, double *D1, double *D2, double *B0r, double *B1, double *B2,
                        int iH)
{
    orc_geom g = *geom_get(c);
    double *D[3] = {D0, D1, D2}, *B[3] = {B0r, B1, B2};
    double *E[3], *H[3];
    for (int k = 0; k < 3; ++k) { E[k] = malloc(g.n * sizeof(double)); H[k] = malloc(g.n * sizeof(double)); }
    aux_fields(&g, D, B, E, H);
    double L = 0.0;
    for (int j = 0; j < c->nth; ++j) {
        double Eth = E[1][IDX(c, iH, j)];
        double Hph = 0.5 * (H[2][IDX(c, iH - 1, j)] + H[2][IDX(c, iH, j)]);
        double Eph = 0.5 * (E[2][IDX(c, iH, j)] + E[2][IDX(c, iH, j + 1)]);
        double Hth = 0.25 * (H[1][IDX(c, iH - 1, j)] + H[1][IDX(c, iH, j)] + H[1][IDX(c, iH - 1, j + 1)] +
                             H[1][IDX(c, iH, j + 1)]);
        L += (Eth * Hph - Eph * Hth) * c->dth;
    }
    for (int k = 0; k < 3; ++k) { free(E[k]); free(H[k]); }
    return L;
}


/* ======================================================================== */
/* 2D radiation and injection (Sec. 4's prescription on the 2D grid, and   */
/* the pair injection of Sec. 3.4's plasma-filled Wald run).                */
/*                                                                          */
/* After the push + deposit, in slot order:                                 */
/*  - a charged massive particle with FIDO Lorentz factor                   */
/*    Gamma = sqrt(1 + gamma^ij u_i u_j) >= gamma_thr (and Gamma - eps_ph   */
/*    >= 1) emits a photon of FIDO energy eps_ph along its momentum and     */
/*    loses that energy: u -> u sqrt((Gamma-eps)^2-1)/sqrt(Gamma^2-1); the  */
/*    photon starts at the emitter with k_i = eps_ph u_i / |u|;             */
/*  - a photon (massless species) with FIDO energy e = |k| > 2 converts     */
/*    with probability 1 - exp(-tau dt): U = uniform(seed, slot, step, 1)   */
/*    < P; it dies and an e- and an e+ start at its position, each with     */
/*    u = s k, s = sqrt((e/2)^2 - 1)/e (FIDO energy e/2 along k).           */
/* Children are appended after all slots, in parent order (photon: one      */
/* child; conversion: e-, then e+).                                         */
/*                                                                          */
/* After the field update, per cell in cell order (c = j nr + i):           */
/*  sigma = B^2 / n with B^2 = gamma_ij B^i B^j and D.B = gamma_ij D^i B^j  */
/*  at the cell centre (x1, x2) = (i + 1/2, j + 1/2) (fields of the shape  */
/*  in use), n = (charged live particles in the cell) |qw_0| / V_cell      */
/*  (V_cell = A^B_phi of the cell, no fewer than one particle); where       */
/*  sigma > sigma_thr and |D.B| / B^2 > eps_db an e- and an e+ are          */
/*  injected at rest in the FIDO frame (u_i = 0) at x = (i + U1, j + U2),  */
/*  U1 = uniform(seed, c, step, 2), U2 = uniform(seed, c, step, 3), appended */
/*  in cell order.                                                          */
/* ======================================================================== */
static double fido_norm2(const orc_metric *m, double u1, double u2, double u3)
{
    return m->gi_rr * u1 * u1 + 2.0 * m->gi_rp * u1 * u3 + m->gi_thth * u2 * u2 + m->gi_pp * u3 * u3;
}

int orc_radiate(const orc_cfg *c, int64_t step, long *np, long cap, double *r, double *th, double *u1, double *u2,
                double *u3, uint32_t *tag, long counts[2])
{
    int status = ORC_OK;
    long n0 = *np, w = n0;
    double P = 1.0 - exp(-c->tau * c->dt);
    counts[0] = counts[1] = 0;
    for (long p = 0; p < n0; ++p) {
        if (tag[p] & ORC_DEAD) continue;
        int sp = tag[p] & 3u;
        orc_metric m;
        metric_at(c->a, r[p], th[p], &m);
        double uu = fido_norm2(&m, u1[p], u2[p], u3[p]);
        if (c->massive[sp] && c->qm[sp] != 0.0) {
            double G = sqrt(1.0 + uu);
            if (G >= c->gamma_thr && G - c->eps_ph >= 1.0) {
                double pm = sqrt(uu), G2 = G - c->eps_ph, f = sqrt(G2 * G2 - 1.0) / pm, k = c->eps_ph / pm;
                double k1 = k * u1[p], k2 = k * u2[p], k3 = k * u3[p];
                u1[p] *= f; u2[p] *= f; u3[p] *= f;
                counts[0]++;
                if (w >= cap) { status = 6; continue; }
                r[w] = r[p]; th[w] = th[p]; u1[w] = k1; u2[w] = k2; u3[w] = k3; tag[w] = 3u;
                ++w;
            }
        } else if (!c->massive[sp]) {
            double e = sqrt(uu);
            if (e > 2.0 && orc_uniform(c->seed, (uint64_t)p, step, 1) < P) {
                double s = sqrt(0.25 * e * e - 1.0) / e;
                tag[p] |= ORC_DEAD;
                counts[1]++;
                for (int k = 0; k < 2; ++k) {
                    if (w >= cap) { status = 6; break; }
                    r[w] = r[p]; th[w] = th[p]; u1[w] = s * u1[p]; u2[w] = s * u2[p]; u3[w] = s * u3[p];
                    tag[w] = (uint32_t)k;
                    ++w;
                }
            }
        }
    }
    *np = w;
    return status;
}

int orc_inject(const orc_cfg *c, int64_t step, long *np, long cap, double *r, double *th, double *u1, double *u2,
               double *u3, uint32_t *tag, double *D0, double *D1, double *D2, double *B0r, double *B1, double *B2,
               long *count)
{
    orc_geom g = *geom_get(c);
    double *D[3] = {D0, D1, D2}, *B[3] = {B0r, B1, B2};
    long ncell = (long)c->nr * c->nth, n0 = *np, w = n0;
    long *nq = calloc(ncell, sizeof(long));
    double lnrin = log(c->r_in);
    for (long p = 0; p < n0; ++p) {
        if (tag[p] & ORC_DEAD) continue;
        int sp = tag[p] & 3u;
        if (!(c->massive[sp] && c->qm[sp] != 0.0)) continue;
        double x1 = (log(r[p]) - lnrin) / c->dx1, x2 = th[p] / c->dth;
        int i = (int)floor(x1), j = jcell(c, x2);
        if (i < 0 || i >= c->nr || j < 0) continue;
        nq[(long)j * c->nr + i]++;
    }
    int status = ORC_OK;
    *count = 0;
    double w0 = fabs(c->qw[0]);
    for (long cc = 0; cc < ncell; ++cc) {
        int i = (int)(cc % c->nr), j = (int)(cc / c->nr);
        double x1 = i + 0.5, x2 = j + 0.5;
        double Dv[3], Bv[3];
        if (c->shape == 3)
            interp_fields3(c, D, B, x1, x2, Dv, Bv);
        else
            interp_fields(c, D, B, x1, x2, Dv, Bv);
        orc_metric m;
        metric_at(c->a, c->r_in * exp(x1 * c->dx1), x2 * c->dth, &m);
        double Bl[3];
        lower(&m, Bv, Bl);
        double B2 = Bl[0] * Bv[0] + Bl[1] * Bv[1] + Bl[2] * Bv[2];
        double DB = Bl[0] * Dv[0] + Bl[1] * Dv[1] + Bl[2] * Dv[2];
        double V = g.AB[2][IDX(c, i, j)];
        double n = (nq[cc] > 0 ? (double)nq[cc] : 1.0) * w0 / V;
        if (!(B2 > 0.0) || !(B2 / n > c->sigma_thr) || !(fabs(DB) / B2 > c->eps_db)) continue;
        double U1 = orc_uniform(c->seed, (uint64_t)cc, step, 2), U2 = orc_uniform(c->seed, (uint64_t)cc, step, 3);
        double rr = c->r_in * exp((i + U1) * c->dx1), tt = (j + U2) * c->dth;
        for (int k = 0; k < 2; ++k) {
            if (w >= cap) { status = 6; break; }
            r[w] = rr; th[w] = tt; u1[w] = 0.0; u2[w] = 0.0; u3[w] = 0.0; tag[w] = (uint32_t)k;
            ++w;
        }
        (*count)++;
    }
    free(nq);
    *np = w;
    return status;
}
