// grpic_init.cu -- start-up kernels: face areas and metric-coefficient tables
// (Sec. 2.1, Eq. area-element: 10-point Gauss quadrature per integrated
// dimension, evaluated once), and the analytic initial fields of App. C.
#include "grpic_internal.cuh"

namespace grpic {
namespace {

struct GL {
    double x[NGL], w[NGL];
};

__device__ double quad_theta(const GridDev &g, const GL &gl, double r, double t0, double t1)
{
    double h = 0.5 * (t1 - t0), m = 0.5 * (t1 + t0), s = 0.0;
#pragma unroll
    for (int k = 0; k < NGL; ++k) s += gl.w[k] * ks_sqrtg(g.a, r, m + h * gl.x[k]);
    return h * s;
}
__device__ double quad_r(const GridDev &g, const GL &gl, double r0, double r1, double th)
{
    double h = 0.5 * (r1 - r0), m = 0.5 * (r1 + r0), s = 0.0;
#pragma unroll
    for (int k = 0; k < NGL; ++k) s += gl.w[k] * ks_sqrtg(g.a, m + h * gl.x[k], th);
    return h * s;
}
__device__ double quad_rt(const GridDev &g, const GL &gl, double r0, double r1, double t0, double t1)
{
    double hr = 0.5 * (r1 - r0), mr = 0.5 * (r1 + r0), ht = 0.5 * (t1 - t0), mt = 0.5 * (t1 + t0), s = 0.0;
    for (int l = 0; l < NGL; ++l) {
        double th = mt + ht * gl.x[l], sl = 0.0;
#pragma unroll
        for (int k = 0; k < NGL; ++k) sl += gl.w[k] * ks_sqrtg(g.a, mr + hr * gl.x[k], th);
        s += gl.w[l] * sl;
    }
    return hr * ht * s;
}

__global__ void tables_kernel(GridDev g, GL gl, double *tab, size_t slab, double *col1d, int damp_cells,
                              double damp_max)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (col >= g.ld_tab || j > g.nth) return;
    int i = col - NG;
    size_t q = (size_t)j * g.ld_tab + col;
    double ri = r_of(g, i), rh = r_of(g, i + 0.5), rml = r_of(g, i - 0.5), rp1 = r_of(g, i + 1.0);
    double tj = j * g.dth, tjh = (j + 0.5) * g.dth, tj1 = (j + 1) * g.dth;
    double tlo = fmax(0.0, (j - 0.5) * g.dth), thi = fmin(M_PI, (j + 0.5) * g.dth);
    bool top = (j == g.nth);

    double adr = quad_theta(g, gl, rh, tlo, thi);
    double adp = quad_rt(g, gl, rml, rh, tlo, thi);
    double abt = quad_r(g, gl, ri, rp1, tj);
    double adt = top ? 0.0 : quad_r(g, gl, rml, rh, tjh);
    double abr = top ? 0.0 : quad_theta(g, gl, ri, tj, tj1);
    double abp = top ? 0.0 : quad_rt(g, gl, ri, rp1, tj, tj1);
    tab[T_ADR * slab + q] = adr;
    tab[T_ADT * slab + q] = adt;
    tab[T_ADP * slab + q] = adp;
    tab[T_ABR * slab + q] = abr;
    tab[T_ABT * slab + q] = abt;
    tab[T_ABP * slab + q] = abp;
    tab[T_INV_ADR * slab + q] = adr > 0 ? 1.0 / adr : 0.0;
    tab[T_INV_ADT * slab + q] = adt > 0 ? 1.0 / adt : 0.0;
    tab[T_INV_ADP * slab + q] = adp > 0 ? 1.0 / adp : 0.0;
    tab[T_INV_ABR * slab + q] = abr > 0 ? 1.0 / abr : 0.0;
    // B^theta on the axis is held at zero: its (vanishing) face gets no inverse
    tab[T_INV_ABT * slab + q] = (j == 0 || top || !(abt > 0)) ? 0.0 : 1.0 / abt;
    tab[T_INV_ABP * slab + q] = abp > 0 ? 1.0 / abp : 0.0;

    KS m;
    // D^r location (i+1/2, j)
    ks_point(g.a, rh, tj, m);
    tab[T_AGRR_DR * slab + q] = m.alpha * m.g_rr;
    tab[T_AGRP_DR * slab + q] = m.alpha * m.g_rp;
    // B^theta location (i+1/2, j)
    tab[T_AGTT_BT * slab + q] = m.alpha * m.g_tt;
    tab[T_SGB_BT * slab + q] = m.sqrtg * m.beta;
    // D^phi location (i, j)
    ks_point(g.a, ri, tj, m);
    tab[T_AGPP_DP * slab + q] = m.alpha * m.g_pp;
    tab[T_AGRP_DP * slab + q] = m.alpha * m.g_rp;
    tab[T_SGB_DP * slab + q] = m.sqrtg * m.beta;
    if (!top) {
        // D^theta and B^r locations (i, j+1/2)
        ks_point(g.a, ri, tjh, m);
        tab[T_AGTT_DT * slab + q] = m.alpha * m.g_tt;
        tab[T_SGB_DT * slab + q] = m.sqrtg * m.beta;
        tab[T_AGRR_BR * slab + q] = m.alpha * m.g_rr;
        tab[T_AGRP_BR * slab + q] = m.alpha * m.g_rp;
        // B^phi location (i+1/2, j+1/2)
        ks_point(g.a, rh, tjh, m);
        tab[T_AGPP_BP * slab + q] = m.alpha * m.g_pp;
        tab[T_AGRP_BP * slab + q] = m.alpha * m.g_rp;
        tab[T_SGB_BP * slab + q] = m.sqrtg * m.beta;
    } else {
        tab[T_AGTT_DT * slab + q] = 0.0;
        tab[T_SGB_DT * slab + q] = 0.0;
        tab[T_AGRR_BR * slab + q] = 0.0;
        tab[T_AGRP_BR * slab + q] = 0.0;
        tab[T_AGPP_BP * slab + q] = 0.0;
        tab[T_AGRP_BP * slab + q] = 0.0;
        tab[T_SGB_BP * slab + q] = 0.0;
    }
    if (j == 0) {
        col1d[0 * g.ld_tab + col] = rp1 - ri;   // primal edge r_{i+1} - r_i
        col1d[1 * g.ld_tab + col] = rh - rml;   // dual edge r_{i+1/2} - r_{i-1/2}
        // outer damping factors 1 - d s^3 at integer and half-integer positions
        double x0 = g.nr - damp_cells;
        double fi = 1.0, fh = 1.0;
        if (damp_cells > 0 && damp_max > 0.0) {
            double si = (i - x0) / damp_cells, sh = (i + 0.5 - x0) / damp_cells;
            if (si > 0.0 && i >= 0 && i <= g.nr) { si = fmin(si, 1.0); fi = 1.0 - damp_max * si * si * si; }
            if (sh > 0.0 && i >= 0 && i <= g.nr - 1) { sh = fmin(sh, 1.0); fh = 1.0 - damp_max * sh * sh * sh; }
        }
        col1d[2 * g.ld_tab + col] = fi;
        col1d[3 * g.ld_tab + col] = fh;
    }
}

// Closed-form fields of App. C: A_t, A_phi, covariant E_i and sqrt(gamma) B^i.
// kind 0 rotating Wald, 1 a=0 Wald (A_phi = B0 gamma_phiphi / 2, E = 0),
// 2 monopole, 3 split monopole (monopole times sgn cos theta).
__device__ void closed_form(int kind, double a, double B0, double r, double th, double &At, double &Aph,
                            double E[3], double sB[3])
{
    double s, c;
    sincos(th, &s, &c);
    double a2 = a * a, r2 = r * r, c2 = c * c, s2 = s * s;
    double rho2 = r2 + a2 * c2;
    double irho2 = 1.0 / rho2, irho4 = irho2 * irho2;
    double Dl = r2 + a2 - 2.0 * r;
    if (kind == 0) {
        // Eqs. wald-vector-potential (t and phi parts unchanged in KS) and wald-solution-ks
        At = B0 * (a * r * (1.0 + c2) * irho2 - a);
        Aph = 0.5 * B0 * s2 * (r2 + a2 - 2.0 * a2 * r * (1.0 + c2) * irho2);
        sB[0] = B0 * (Dl + 2.0 * r * (r2 * r2 - a2 * a2) * irho4) * s * c;
        sB[1] = -B0 * (r + a2 * (1.0 + c2) * (2.0 * r2 - rho2) * irho4) * s2;
        sB[2] = -B0 * (2.0 * a * r * (a2 - r2) * irho4 - a) * s * c;
        E[0] = B0 * a * (1.0 + c2) * (a2 * c2 - r2) * irho4;
        E[1] = 2.0 * B0 * a * r * (a2 - r2) * s * c * irho4;
        E[2] = 0.0;
    } else if (kind == 1) {
        // gamma_phiphi = Sigma sin^2 / rho^2 and its derivatives
        double Sg = (r2 + a2) * (r2 + a2) - a2 * Dl * s2;
        double dSr = 4.0 * r * (r2 + a2) - a2 * (2.0 * r - 2.0) * s2;
        double dSt = -2.0 * a2 * Dl * s * c;
        double gpp = Sg * s2 * irho2;
        double dgr = (dSr * s2 - Sg * s2 * 2.0 * r * irho2) * irho2;
        double dgt = (dSt * s2 + 2.0 * Sg * s * c + Sg * s2 * 2.0 * a2 * c * s * irho2) * irho2;
        At = 0.0;
        Aph = 0.5 * B0 * gpp;
        sB[0] = 0.5 * B0 * dgt;
        sB[1] = -0.5 * B0 * dgr;
        sB[2] = 0.0;
        E[0] = E[1] = E[2] = 0.0;
    } else {
        double sg = 1.0;
        if (kind == 3) sg = c > 0.0 ? 1.0 : (c < 0.0 ? -1.0 : 0.0);
        double f = sg * B0;
        At = f * a * c * irho2;
        Aph = -f * c * (r2 + a2) * irho2;
        sB[0] = f * (a2 + r2) * (r2 - a2 * c2) * s * irho4;
        sB[1] = -f * 2.0 * a2 * r * s2 * c * irho4;
        sB[2] = f * a * (r2 - a2 * c2) * s * irho4;
        E[0] = -f * 2.0 * a * r * c * irho4;
        E[1] = -f * a * (r2 - a2 * c2) * s * irho4;
        E[2] = 0.0;
    }
}

// D^j = gamma^{ji} (E_i - e_ikl beta^k B^l) / alpha (Eq. E-H-B-D solved for D)
__device__ void closed_D(int kind, double a, double B0, double r, double th, double D[3])
{
    double At, Aph, E[3], sB[3];
    closed_form(kind, a, B0, r, th, At, Aph, E, sB);
    KS m;
    ks_point(a, r, th, m);
    double Et = E[1] + m.beta * sB[2];   // - e_{th r ph} beta B^ph
    double Ep = E[2] - m.beta * sB[1];   // - e_{ph r th} beta B^th
    double ia = 1.0 / m.alpha;
    D[0] = (m.gi_rr * E[0] + m.gi_rp * Ep) * ia;
    D[1] = m.gi_tt * Et * ia;
    D[2] = (m.gi_rp * E[0] + m.gi_pp * Ep) * ia;
}

__device__ double aphi(int kind, double a, double B0, double r, double th)
{
    double At, Aph, E[3], sB[3];
    closed_form(kind, a, B0, r, th, At, Aph, E, sB);
    return Aph;
}

template <typename T>
__global__ void init_fields_kernel(GridDev g, GL gl, int kind, double B0, const double *tab, size_t slab, T *D0, T *D1,
                                   T *D2, T *B0r, T *B1, T *B2, T *J0, T *J1, T *J2, int64_t ld)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (col >= g.ld_tab || j > g.nth) return;
    int i = col - NG;
    size_t q = (size_t)j * ld + col, qt = (size_t)j * g.ld_tab + col;
    double ri = r_of(g, i), rp1 = r_of(g, i + 1.0), rh = r_of(g, i + 0.5);
    double tj = j * g.dth, tj1 = (j + 1) * g.dth, tjh = (j + 0.5) * g.dth;
    double br = 0.0, bt = 0.0, bp = 0.0, dr = 0.0, dt = 0.0, dp = 0.0, D[3];
    if (j < g.nth) {
        // Stokes: B^r A^B_r = A_phi(r_i, th_{j+1}) - A_phi(r_i, th_j)
        br = (aphi(kind, g.a, B0, ri, tj1) - aphi(kind, g.a, B0, ri, tj)) * tab[T_INV_ABR * slab + qt];
        // face average of the closed-form B^phi
        double hr = 0.5 * (rp1 - ri), mr = 0.5 * (rp1 + ri), ht = 0.5 * g.dth, mt = tjh, s = 0.0;
        for (int l = 0; l < NGL; ++l) {
            double sl = 0.0;
            for (int k = 0; k < NGL; ++k) {
                double At, Aph, E[3], sB[3];
                closed_form(kind, g.a, B0, mr + hr * gl.x[k], mt + ht * gl.x[l], At, Aph, E, sB);
                sl += gl.w[k] * sB[2];
            }
            s += gl.w[l] * sl;
        }
        bp = hr * ht * s * tab[T_INV_ABP * slab + qt];
        closed_D(kind, g.a, B0, ri, tjh, D);
        dt = D[1];
    }
    if (j > 0 && j < g.nth) {
        // Stokes: B^th A^B_th = -(A_phi(r_{i+1}, th_j) - A_phi(r_i, th_j))
        bt = -(aphi(kind, g.a, B0, rp1, tj) - aphi(kind, g.a, B0, ri, tj)) * tab[T_INV_ABT * slab + qt];
        closed_D(kind, g.a, B0, ri, tj, D);
        dp = D[2];
    }
    closed_D(kind, g.a, B0, rh, tj, D);
    dr = D[0];
    D0[q] = (T)dr;
    D1[q] = (T)dt;
    D2[q] = (T)dp;
    B0r[q] = (T)br;
    B1[q] = (T)bt;
    B2[q] = (T)bp;
    J0[q] = (T)0;
    J1[q] = (T)0;
    J2[q] = (T)0;
}

// guard copies (zero derivative at r_in; same at the outer edge) and the axis
// values D^phi = B^theta = 0 (Sec. 2.1); one thread per row
template <typename T>
__global__ void bc_kernel(GridDev g, T *D0, T *D1, T *D2, T *B0r, T *B1, T *B2, int64_t ld)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > g.nth) return;
    T *half_r[3] = {D0, B1, B2};
    T *int_r[3] = {D1, D2, B0r};
    size_t row = (size_t)j * ld;
    for (int k = 0; k < 3; ++k) {
        for (int c = 0; c < NG; ++c) {
            half_r[k][row + c] = half_r[k][row + NG];
            int_r[k][row + c] = int_r[k][row + NG];
        }
        for (int c = NG + g.nr; c < g.ld_tab; ++c) half_r[k][row + c] = half_r[k][row + NG + g.nr - 1];
        for (int c = NG + g.nr + 1; c < g.ld_tab; ++c) int_r[k][row + c] = int_r[k][row + NG + g.nr];
    }
    if (j == 0 || j == g.nth) {
        for (int c = 0; c < g.ld_tab; ++c) {
            D2[row + c] = (T)0;
            B1[row + c] = (T)0;
        }
    }
}

GL make_gl(const grpic_ctx *ctx)
{
    GL gl;
    for (int k = 0; k < NGL; ++k) {
        gl.x[k] = ctx->gl_x[k];
        gl.w[k] = ctx->gl_w[k];
    }
    return gl;
}

}  // namespace

cudaError_t launch_tables(grpic_ctx *ctx, cudaStream_t s)
{
    dim3 blk(32, 4), grd((ctx->g.ld_tab + 31) / 32, (ctx->g.nth + 1 + 3) / 4);
    tables_kernel<<<grd, blk, 0, s>>>(ctx->g, make_gl(ctx), ctx->tab, ctx->slab, ctx->col1d, ctx->grid.damp_cells,
                                      ctx->grid.damp_max);
    return cudaGetLastError();
}

// the tables of spin a (grid unchanged) into caller buffers: the spin
// gradient differences them at a +- h
cudaError_t launch_tables_at(grpic_ctx *ctx, double a, double *tab, double *col1d, cudaStream_t s)
{
    GridDev g = ctx->g;
    g.a = a;
    dim3 blk(32, 4), grd((ctx->g.ld_tab + 31) / 32, (ctx->g.nth + 1 + 3) / 4);
    tables_kernel<<<grd, blk, 0, s>>>(g, make_gl(ctx), tab, ctx->slab, col1d, ctx->grid.damp_cells,
                                      ctx->grid.damp_max);
    return cudaGetLastError();
}

cudaError_t launch_init_fields_at(grpic_ctx *ctx, double a, const double *tab, int kind, double B0,
                                  const grpic_fields *f, cudaStream_t s)
{
    GridDev g = ctx->g;
    g.a = a;
    dim3 blk(32, 4), grd((ctx->g.ld_tab + 31) / 32, (ctx->g.nth + 1 + 3) / 4);
    int rows = ctx->g.nth + 1;
    double *D[3], *B[3], *J[3];
    for (int k = 0; k < 3; ++k) {
        D[k] = (double *)f->D[k];
        B[k] = (double *)f->B[k];
        J[k] = (double *)f->J[k];
    }
    init_fields_kernel<double><<<grd, blk, 0, s>>>(g, make_gl(ctx), kind, B0, tab, ctx->slab, D[0], D[1], D[2], B[0],
                                                   B[1], B[2], J[0], J[1], J[2], f->ld);
    bc_kernel<double><<<(rows + 127) / 128, 128, 0, s>>>(g, D[0], D[1], D[2], B[0], B[1], B[2], f->ld);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(grpic_ctx *ctx, int kind, double B0, const grpic_fields *f, cudaStream_t s)
{
    dim3 blk(32, 4), grd((ctx->g.ld_tab + 31) / 32, (ctx->g.nth + 1 + 3) / 4);
    int rows = ctx->g.nth + 1;
    if (ctx->prm.precision == 64) {
        double *D[3], *B[3], *J[3];
        for (int k = 0; k < 3; ++k) {
            D[k] = (double *)f->D[k];
            B[k] = (double *)f->B[k];
            J[k] = (double *)f->J[k];
        }
        init_fields_kernel<double><<<grd, blk, 0, s>>>(ctx->g, make_gl(ctx), kind, B0, ctx->tab, ctx->slab, D[0], D[1],
                                                       D[2], B[0], B[1], B[2], J[0], J[1], J[2], f->ld);
        bc_kernel<double><<<(rows + 127) / 128, 128, 0, s>>>(ctx->g, D[0], D[1], D[2], B[0], B[1], B[2], f->ld);
    } else {
        float *D[3], *B[3], *J[3];
        for (int k = 0; k < 3; ++k) {
            D[k] = (float *)f->D[k];
            B[k] = (float *)f->B[k];
            J[k] = (float *)f->J[k];
        }
        init_fields_kernel<float><<<grd, blk, 0, s>>>(ctx->g, make_gl(ctx), kind, B0, ctx->tab, ctx->slab, D[0], D[1],
                                                      D[2], B[0], B[1], B[2], J[0], J[1], J[2], f->ld);
        bc_kernel<float><<<(rows + 127) / 128, 128, 0, s>>>(ctx->g, D[0], D[1], D[2], B[0], B[1], B[2], f->ld);
    }
    return cudaGetLastError();
}

}  // namespace grpic
