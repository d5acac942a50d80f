// grpic_adjoint.cu -- the differentiable form: a hand-written adjoint of the
// FP64 time step (push + deposit + field update, arXiv:2503.04558 Sec. 2) for
// the time-averaged radial Poynting flux through the horizon ring,
//   L = (1/N) sum_n sum_j (E_th H_ph - E_ph H_th)(i_H, j+1/2) dtheta,
// with respect to the initial particle state and the initial fields.
//
// Reverse sweep per step n (state S_n = particles, F_n = D, B):
//   * seed   lambda_F^{n+1} += dL/dF^{n+1}  (through the auxiliary fields);
//   * fields the field update is linear in (F^n, J): its transpose runs the
//            predictor-corrector stages backwards with the transposed circulation
//            and auxiliary-field stencils (scatter with atomics), the boundary
//            copies transposed into their source cells;
//   * particles for every particle: the transpose of the deposit (derivatives of
//            the piecewise-linear CIC weights), the axis reflection, the geodesic
//            step (the predictor and correctors as run, transposed one by one,
//            or the implicit-function theorem at the converged trapezoid,
//            (I - dt/2 dF/dy)^T w = lambda, a 5x5 solve), the Boris step and the
//            interpolation (scatter of lambda_E into lambda_F).  Vector-Jacobian
//            products of the right-hand side are a hand-written reverse pass;
//            the metric's derivatives and the other local Jacobians come from
//            forward-mode dual numbers through the same metric code.
// Recompute checkpoints every `checkpoint_every` steps bound the memory; the
// segment's recompute runs the FP64 push in its recording form, so the
// particle adjoint reads the Boris output and the corrector iterates (with
// sin, cos of theta) instead of running the push again.
#include "grpic_geo.cuh"

#include <cstring>
#include <new>
#include <vector>

namespace grpic {

// ---- forward-mode dual numbers ---------------------------------------------
template <int N>
struct DN {
    double v;
    double d[N];
    __device__ DN() {}
    __device__ DN(double x) : v(x)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = 0.0;
    }
};
template <int N>
__device__ __forceinline__ DN<N> operator+(const DN<N> &a, const DN<N> &b)
{
    DN<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ DN<N> operator-(const DN<N> &a, const DN<N> &b)
{
    DN<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ DN<N> operator-(const DN<N> &a)
{
    DN<N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ DN<N> operator*(const DN<N> &a, const DN<N> &b)
{
    DN<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N>
__device__ __forceinline__ DN<N> operator/(const DN<N> &a, const DN<N> &b)
{
    DN<N> r;
    double ib = rcp_t(b.v);
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <int N>
__device__ __forceinline__ DN<N> rcp_t(const DN<N> &a)
{
    DN<N> r;
    r.v = rcp_t(a.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k] * r.v * r.v;
    return r;
}
template <int N>
__device__ __forceinline__ DN<N> sqrt_t(const DN<N> &a)
{
    DN<N> r;
    r.v = sqrt_t(a.v);
    double h = a.v > 0.0 ? 0.5 * rcp_t(r.v) : 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
    return r;
}
template <int N>
__device__ __forceinline__ void sincos_t(const DN<N> &a, DN<N> *s, DN<N> *c)
{
    double sv, cv;
    sincos(a.v, &sv, &cv);
    s->v = sv;
    c->v = cv;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        s->d[k] = cv * a.d[k];
        c->d[k] = -sv * a.d[k];
    }
}

namespace {

// ---- the particle's local maps ---------------------------------------------
// right-hand side of Eq. particle-eom (no Lorentz force) at y = (r, th, ur, ut, up)
template <typename T>
__device__ __forceinline__ void rhs_y(double a, double eps, const T y[5], T f[6])
{
    T s, c;
    sincos_t(y[1], &s, &c);
    KSGeo<T> m;
    ks_geo_sc<T>(T(a), y[0], s, c, m);
    RhsT<T> o;
    geo_rhs_m<T, T>(m, T(eps), y[2], y[3], y[4], o);
    f[0] = o.xr;
    f[1] = o.xt;
    f[2] = o.xp;
    f[3] = o.ur;
    f[4] = o.ut;
    f[5] = T(0.0);
}

// F = (X^r, X^th, U_r, U_th, U_ph) and X^ph at y, with dF/dy and dX^ph/dy
__device__ void rhs_jac(double a, double eps, const double y[5], double F[5], double J[5][5], double &Fp,
                        double dFp[5])
{
    DN<5> yd[5], f[6];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        yd[k] = DN<5>(y[k]);
        yd[k].d[k] = 1.0;
    }
    rhs_y<DN<5>>(a, eps, yd, f);
    const int map[5] = {0, 1, 3, 4, 5};
    for (int r = 0; r < 5; ++r) {
        F[r] = f[map[r]].v;
        for (int k = 0; k < 5; ++k) J[r][k] = f[map[r]].d[k];
    }
    Fp = f[2].v;
    for (int k = 0; k < 5; ++k) dFp[k] = f[2].d[k];
}

// w^T dF/dy + wp dX^ph/dy at y = (r, th, u_r, u_th, u_ph) for F = (X^r, X^th,
// U_r, U_th, 0), the right-hand side of Eq. particle-eom written as the push
// evaluates it: with P = (a^2 + r^2) u_r^2 + 2 a u_r u_ph + u_th^2 +
// u_ph^2 / sin^2,  u.u = P / rho^2 - beta u_r^2,  X^r = (g^rr u_r + g^rph u_ph)
// / u^0 - beta,  Q_r = u_r^2 (z - d_r beta) - 2 r P / rho^4,  Q_th = -d_th rho^2
// P / rho^4 - d_th beta u_r^2 - 2 sin cos u_ph^2 / (rho^2 sin^4),  U_i =
// -alpha u^0 d_i alpha + u_r d_i beta - Q_i / (2 u^0).  The reverse pass runs
// through those formulas; the r, theta (and a) derivatives of the thirteen
// metric quantities they use come from dual numbers.  sv, cv = sin, cos y[1].
template <int ND>
__device__ void rhs_vjp_p(double a, double eps, const double y[5], double sv, double cv, const double w[5], double wp,
                          double out[5], double *out_a = nullptr)
{
    typedef DN<ND> D;
    D r(y[0]), aD(a), s(sv), c(cv);
    r.d[0] = 1.0;
    s.d[1] = cv;
    c.d[1] = -sv;
    if constexpr (ND > 2) aD.d[2] = 1.0;
    // metric quantities (dual)
    const D a2 = aD * aD, r2 = r * r;
    const D A2 = a2 + r2;
    const D ir = rcp_t(r2 + a2 * c * c);
    const D ir2 = ir * ir;
    const D z = D(2.0) * r * ir;
    const D iopz = rcp_t(D(1.0) + z);
    const D alphaD = sqrt_t(iopz);
    const D betaD = z * iopz;
    const D is2 = rcp_t(s * s);
    const D drho_t = D(-2.0) * a2 * c * s;
    const D dz_r = D(2.0) * ir * (D(1.0) - D(2.0) * r2 * ir);
    const D dz_t = D(-2.0) * r * drho_t * ir2;
    const D ka = D(-0.5) * alphaD * iopz, kb = iopz * iopz;
    const D da_r = ka * dz_r, da_t = ka * dz_t, db_r = kb * dz_r, db_t = kb * dz_t;
    const D M2 = D(2.0) * r * ir2, M3 = drho_t * ir2, M4 = D(2.0) * s * c * ir * is2 * is2;
    // forward values
    const double ur = y[2], ut = y[3], up = y[4];
    const double vA2 = A2.v, vir = ir.v, vbe = betaD.v, val = alphaD.v, vis2 = is2.v, vz = z.v;
    const double ur2 = ur * ur, up2 = up * up;
    const double P = vA2 * ur2 + 2.0 * a * ur * up + ut * ut + vis2 * up2;
    const double uu = vir * P - vbe * ur2;
    const double au0 = sqrt_t(eps + uu);
    const double iau = rcp_t(au0);
    const double iu0 = val * iau, h = 0.5 * iu0;
    const double G1 = vA2 * vir - vbe, G2 = a * vir;
    const double Qr = ur2 * (vz - db_r.v) - M2.v * P;
    const double Qt = -M3.v * P - db_t.v * ur2 - M4.v * up2;
    // reverse; adjoints of the outputs X^r, X^th, U_r, U_th, X^ph
    const double Lxr = w[0], Lxt = w[1], Lur = w[2], Lut = w[3], Lxp = wp;
    double L_ur = 0.0, L_ut = 0.0, L_up = 0.0, L_a = 0.0;
    double L_A2 = 0.0, L_ir = 0.0, L_be = 0.0, L_al = 0.0, L_is2 = 0.0, L_z = 0.0;
    double L_dar = 0.0, L_dat = 0.0, L_dbr = 0.0, L_dbt = 0.0, L_M2 = 0.0, L_M3 = 0.0, L_M4 = 0.0;
    double L_au0 = 0.0, L_iu0 = 0.0, L_P = 0.0;
    // U_r = -au0 da_r + ur db_r - h Qr,  U_th likewise
    L_au0 -= Lur * da_r.v + Lut * da_t.v;
    L_dar -= Lur * au0;
    L_dat -= Lut * au0;
    L_dbr += Lur * ur;
    L_dbt += Lut * ur;
    L_ur += Lur * db_r.v + Lut * db_t.v;
    const double L_h = -Lur * Qr - Lut * Qt;
    const double L_Qr = -Lur * h, L_Qt = -Lut * h;
    // Qr = ur^2 (z - db_r) - M2 P
    L_ur += L_Qr * 2.0 * ur * (vz - db_r.v);
    L_z += L_Qr * ur2;
    L_dbr -= L_Qr * ur2;
    L_M2 -= L_Qr * P;
    L_P -= L_Qr * M2.v;
    // Qt = -M3 P - db_t ur^2 - M4 up^2
    L_M3 -= L_Qt * P;
    L_P -= L_Qt * M3.v;
    L_dbt -= L_Qt * ur2;
    L_ur -= L_Qt * 2.0 * db_t.v * ur;
    L_M4 -= L_Qt * up2;
    L_up -= L_Qt * 2.0 * M4.v * up;
    // h = iu0 / 2
    L_iu0 += 0.5 * L_h;
    // X^r = (G1 ur + G2 up) iu0 - beta, G1 = A2 ir - beta, G2 = a ir
    L_iu0 += Lxr * (G1 * ur + G2 * up);
    L_ur += Lxr * G1 * iu0;
    L_up += Lxr * G2 * iu0;
    L_A2 += Lxr * ur * iu0 * vir;
    L_ir += Lxr * iu0 * (ur * vA2 + a * up);
    L_be -= Lxr * (ur * iu0 + 1.0);
    L_a += Lxr * vir * up * iu0;
    // X^th = ir ut iu0
    L_iu0 += Lxt * vir * ut;
    L_ut += Lxt * vir * iu0;
    L_ir += Lxt * ut * iu0;
    // X^ph = (a ir ur + ir is2 up) iu0
    L_iu0 += Lxp * (a * vir * ur + vir * vis2 * up);
    L_ur += Lxp * a * vir * iu0;
    L_up += Lxp * vir * vis2 * iu0;
    L_ir += Lxp * (a * ur + vis2 * up) * iu0;
    L_is2 += Lxp * vir * up * iu0;
    L_a += Lxp * vir * ur * iu0;
    // iu0 = alpha / au0, au0 = sqrt(eps + uu)
    L_al += L_iu0 * iau;
    L_au0 -= L_iu0 * val * iau * iau;
    const double L_uu = 0.5 * L_au0 * iau;
    // uu = ir P - beta ur^2
    L_ir += L_uu * P;
    L_P += L_uu * vir;
    L_be -= L_uu * ur2;
    L_ur -= L_uu * 2.0 * vbe * ur;
    // P = A2 ur^2 + 2 a ur up + ut^2 + is2 up^2
    L_A2 += L_P * ur2;
    L_ur += L_P * (2.0 * vA2 * ur + 2.0 * a * up);
    L_up += L_P * (2.0 * a * ur + 2.0 * vis2 * up);
    L_ut += L_P * 2.0 * ut;
    L_is2 += L_P * up2;
    L_a += L_P * 2.0 * ur * up;
    // metric quantities -> r, theta (and a)
    const D *q[13] = {&A2, &ir, &betaD, &alphaD, &is2, &z, &da_r, &da_t, &db_r, &db_t, &M2, &M3, &M4};
    const double Lq[13] = {L_A2, L_ir, L_be, L_al, L_is2, L_z, L_dar, L_dat, L_dbr, L_dbt, L_M2, L_M3, L_M4};
    double Lr = 0.0, Lth = 0.0;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        Lr += Lq[k] * q[k]->d[0];
        Lth += Lq[k] * q[k]->d[1];
    }
    if constexpr (ND > 2) {
        double La = L_a;
#pragma unroll
        for (int k = 0; k < 13; ++k) La += Lq[k] * q[k]->d[2];
        *out_a += La;
    }
    out[0] = Lr;
    out[1] = Lth;
    out[2] = L_ur;
    out[3] = L_ut;
    out[4] = L_up;
}

// lo^T d(u')/dz for the generalized Boris step (Eqs. boris-plus-minus, u0bar,
// boris-scheme) u' = u'(z), z = (r, th, u_r, u_th, u_ph, D^r, D^th, D^ph, B^r,
// B^th, B^ph): its reverse pass written out by hand, the metric's r and theta
// derivatives from two-slot dual numbers; sn, cs = sin, cos of theta
template <int ND>
__device__ void boris_vjp(double a, double qm, double dt, const double z[11], double sn, double cs, const double lo[3],
                          double out[11], double *out_a = nullptr)
{
    // slots: d/dr, d/dtheta (and d/da when ND = 3)
    DN<ND> r(z[0]), aD(a), s(sn), c(cs);
    r.d[0] = 1.0;
    s.d[1] = cs;
    c.d[1] = -sn;
    if constexpr (ND > 2) aD.d[2] = 1.0;
    const DN<ND> a2 = aD * aD, s2 = s * s;
    const DN<ND> rho2 = r * r + a2 * c * c;
    const DN<ND> ir = rcp_t(rho2);
    const DN<ND> zz = DN<ND>(2.0) * r * ir;
    const DN<ND> opz = DN<ND>(1.0) + zz;
    const DN<ND> alphaD = sqrt_t(rcp_t(opz));
    const DN<ND> Dl_ = r * r + a2 - DN<ND>(2.0) * r;
    const DN<ND> Sg = (r * r + a2) * (r * r + a2) - a2 * Dl_ * s2;
    // metric quantities q[] = g_rr, g_rp, g_tt, g_pp, i_rr, i_rp, i_tt, i_pp, sqrt(gamma), alpha
    DN<ND> q[10];
    q[0] = opz;
    q[1] = -aD * s2 * opz;
    q[2] = rho2;
    q[3] = Sg * s2 * ir;
    q[4] = (a2 + r * r) * ir - zz * rcp_t(opz);
    q[5] = aD * ir;
    q[6] = ir;
    q[7] = ir * rcp_t(s2);
    q[8] = rho2 * s * sqrt_t(opz);
    q[9] = alphaD;
    const double grr = q[0].v, grp = q[1].v, gtt = q[2].v, gpp = q[3].v;
    const double irr = q[4].v, irp = q[5].v, itt = q[6].v, ipp = q[7].v, sg = q[8].v, alpha = q[9].v;
    const double u[3] = {z[2], z[3], z[4]}, D[3] = {z[5], z[6], z[7]}, B[3] = {z[8], z[9], z[10]};
    const double c1 = 0.5 * qm * dt;
    // forward values
    const double Dl[3] = {grr * D[0] + grp * D[2], gtt * D[1], grp * D[0] + gpp * D[2]};
    const double h = c1 * alpha;
    const double um[3] = {u[0] + h * Dl[0], u[1] + h * Dl[1], u[2] + h * Dl[2]};
    const double v[3] = {irr * um[0] + irp * um[2], itt * um[1], irp * um[0] + ipp * um[2]};
    const double S = 1.0 + um[0] * v[0] + um[1] * v[1] + um[2] * v[2];
    const double rS = sqrt_t(S);
    const double ialpha = rcp_t(alpha), irS = rcp_t(rS);
    const double u0b = rS * ialpha;
    const double iu0b = alpha * irS;
    const double kt = c1 * iu0b;
    const double t[3] = {kt * B[0], kt * B[1], kt * B[2]};
    const double Gt[3] = {grr * t[0] + grp * t[2], gtt * t[1], grp * t[0] + gpp * t[2]};
    const double tt = t[0] * Gt[0] + t[1] * Gt[1] + t[2] * Gt[2];
    const double i1tt = rcp_t(1.0 + tt);
    const double ks = 2.0 * i1tt;
    const double sv[3] = {ks * t[0], ks * t[1], ks * t[2]};
    const double vt[3] = {v[1] * t[2] - v[2] * t[1], v[2] * t[0] - v[0] * t[2], v[0] * t[1] - v[1] * t[0]};
    const double w[3] = {um[0] + sg * vt[0], um[1] + sg * vt[1], um[2] + sg * vt[2]};
    const double x[3] = {irr * w[0] + irp * w[2], itt * w[1], irp * w[0] + ipp * w[2]};
    const double C[3] = {x[1] * sv[2] - x[2] * sv[1], x[2] * sv[0] - x[0] * sv[2], x[0] * sv[1] - x[1] * sv[0]};
    // reverse: out_i = um_i + sg C_i + h Dl_i
    double Lum[3] = {lo[0], lo[1], lo[2]};
    double Lh = lo[0] * Dl[0] + lo[1] * Dl[1] + lo[2] * Dl[2];
    double LDl[3] = {lo[0] * h, lo[1] * h, lo[2] * h};
    double Lq[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    Lq[8] += lo[0] * C[0] + lo[1] * C[1] + lo[2] * C[2];
    const double LC[3] = {lo[0] * sg, lo[1] * sg, lo[2] * sg};
    // C = x cross s
    double Lx[3] = {sv[1] * LC[2] - sv[2] * LC[1], sv[2] * LC[0] - sv[0] * LC[2], sv[0] * LC[1] - sv[1] * LC[0]};
    double Ls[3] = {LC[1] * x[2] - LC[2] * x[1], LC[2] * x[0] - LC[0] * x[2], LC[0] * x[1] - LC[1] * x[0]};
    // x = Ginv w
    double Lw[3] = {irr * Lx[0] + irp * Lx[2], itt * Lx[1], irp * Lx[0] + ipp * Lx[2]};
    Lq[4] += Lx[0] * w[0];
    Lq[5] += Lx[0] * w[2] + Lx[2] * w[0];
    Lq[6] += Lx[1] * w[1];
    Lq[7] += Lx[2] * w[2];
    // w = um + sg (v cross t)
    for (int i = 0; i < 3; ++i) Lum[i] += Lw[i];
    Lq[8] += Lw[0] * vt[0] + Lw[1] * vt[1] + Lw[2] * vt[2];
    const double LD_[3] = {Lw[0] * sg, Lw[1] * sg, Lw[2] * sg};
    double Lv[3] = {t[1] * LD_[2] - t[2] * LD_[1], t[2] * LD_[0] - t[0] * LD_[2], t[0] * LD_[1] - t[1] * LD_[0]};
    double Lt[3] = {LD_[1] * v[2] - LD_[2] * v[1], LD_[2] * v[0] - LD_[0] * v[2], LD_[0] * v[1] - LD_[1] * v[0]};
    // s = ks t, ks = 2 / (1 + tt), tt = t^T G t
    const double Lks = Ls[0] * t[0] + Ls[1] * t[1] + Ls[2] * t[2];
    for (int i = 0; i < 3; ++i) Lt[i] += ks * Ls[i];
    const double Ltt = -Lks * 2.0 * i1tt * i1tt;
    for (int i = 0; i < 3; ++i) Lt[i] += 2.0 * Ltt * Gt[i];
    Lq[0] += Ltt * t[0] * t[0];
    Lq[1] += Ltt * 2.0 * t[0] * t[2];
    Lq[2] += Ltt * t[1] * t[1];
    Lq[3] += Ltt * t[2] * t[2];
    // t = kt B, kt = c1 / u0b, u0b = sqrt(S) / alpha
    const double Lkt = Lt[0] * B[0] + Lt[1] * B[1] + Lt[2] * B[2];
    const double LB[3] = {kt * Lt[0], kt * Lt[1], kt * Lt[2]};
    const double Lu0b = -Lkt * c1 * iu0b * iu0b;
    const double LS = 0.5 * Lu0b * irS * ialpha;
    Lq[9] -= Lu0b * rS * ialpha * ialpha;
    // S = 1 + um . v, v = Ginv um
    for (int i = 0; i < 3; ++i) {
        Lum[i] += LS * v[i];
        Lv[i] += LS * um[i];
    }
    Lum[0] += irr * Lv[0] + irp * Lv[2];
    Lum[1] += itt * Lv[1];
    Lum[2] += irp * Lv[0] + ipp * Lv[2];
    Lq[4] += Lv[0] * um[0];
    Lq[5] += Lv[0] * um[2] + Lv[2] * um[0];
    Lq[6] += Lv[1] * um[1];
    Lq[7] += Lv[2] * um[2];
    // um = u + h Dl, h = c1 alpha, Dl = G D
    for (int i = 0; i < 3; ++i) {
        Lh += Lum[i] * Dl[i];
        LDl[i] += h * Lum[i];
    }
    Lq[9] += c1 * Lh;
    const double LDv[3] = {grr * LDl[0] + grp * LDl[2], gtt * LDl[1], grp * LDl[0] + gpp * LDl[2]};
    Lq[0] += LDl[0] * D[0];
    Lq[1] += LDl[0] * D[2] + LDl[2] * D[0];
    Lq[2] += LDl[1] * D[1];
    Lq[3] += LDl[2] * D[2];
    double Lr = 0.0, Lth = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        Lr += Lq[k] * q[k].d[0];
        Lth += Lq[k] * q[k].d[1];
    }
    if constexpr (ND > 2) {
        double La = 0.0;
#pragma unroll
        for (int k = 0; k < 10; ++k) La += Lq[k] * q[k].d[2];
        *out_a += La;
    }
    out[0] = Lr;
    out[1] = Lth;
    for (int i = 0; i < 3; ++i) {
        out[2 + i] = Lum[i];
        out[5 + i] = LDv[i];
        out[8 + i] = LB[i];
    }
}

// small dense solve M x = b (n = 5), Gaussian elimination with partial pivoting
__device__ void solve5(double M[5][5], double b[5])
{
    for (int c = 0; c < 5; ++c) {
        int p = c;
        for (int r = c + 1; r < 5; ++r)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (p != c) {
            for (int k = 0; k < 5; ++k) {
                double t = M[c][k];
                M[c][k] = M[p][k];
                M[p][k] = t;
            }
            double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        double iv = 1.0 / M[c][c];
        for (int r = c + 1; r < 5; ++r) {
            double f = M[r][c] * iv;
            for (int k = c; k < 5; ++k) M[r][k] -= f * M[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int c = 4; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < 5; ++k) s -= M[c][k] * b[k];
        b[c] = s / M[c][c];
    }
}

__device__ __forceinline__ double W1(double d)
{
    d = fabs(d);
    return d < 1.0 ? 1.0 - d : 0.0;
}
__device__ __forceinline__ double dW1(double d) { return fabs(d) < 1.0 ? (d > 0.0 ? -1.0 : (d < 0.0 ? 1.0 : 0.0)) : 0.0; }

__device__ __forceinline__ int jcell(const GridDev &g, double x2)
{
    int j = (int)floor(x2);
    return j > g.nth - 1 ? g.nth - 1 : j;
}

// staggered bilinear stencil with axis mirroring (as in the push)
struct St {
    int c0, r0, r1;
    double f, gg, p0, p1;
};
__device__ __forceinline__ void stencil(const GridDev &g, double x1, double x2, bool half_r, bool half_t, double par,
                                        St &S)
{
    double xi = half_r ? x1 - 0.5 : x1;
    double fi = floor(xi);
    S.f = xi - fi;
    S.c0 = (int)fi + NG;
    S.p0 = S.p1 = 1.0;
    if (half_t) {
        double eta = x2 - 0.5, fj = floor(eta);
        int j = (int)fj;
        S.gg = eta - fj;
        S.r0 = j;
        S.r1 = j + 1;
        if (S.r0 < 0) { S.r0 = -1 - S.r0; S.p0 = par; }
        if (S.r1 > g.nth - 1) { S.r1 = 2 * g.nth - 1 - S.r1; S.p1 = par; }
    } else {
        int j = (int)floor(x2);
        if (j > g.nth - 1) j = g.nth - 1;
        S.gg = x2 - j;
        S.r0 = j;
        S.r1 = j + 1;
    }
}
// value and d/dx1, d/dx2 (logical) of the interpolant
__device__ __forceinline__ void gather_d(const double *F, int64_t ld, const St &S, double &v, double &d1, double &d2)
{
    double a00 = S.p0 * F[(size_t)S.r0 * ld + S.c0], a10 = S.p0 * F[(size_t)S.r0 * ld + S.c0 + 1];
    double a01 = S.p1 * F[(size_t)S.r1 * ld + S.c0], a11 = S.p1 * F[(size_t)S.r1 * ld + S.c0 + 1];
    double f = S.f, g = S.gg;
    v = (1 - f) * (1 - g) * a00 + f * (1 - g) * a10 + (1 - f) * g * a01 + f * g * a11;
    d1 = (1 - g) * (a10 - a00) + g * (a11 - a01);
    d2 = (1 - f) * (a01 - a00) + f * (a11 - a10);
}
__device__ __forceinline__ void scatter_w(double *L, int64_t ld, const St &S, double lam)
{
    double f = S.f, g = S.gg;
    atomicAdd(L + (size_t)S.r0 * ld + S.c0, S.p0 * (1 - f) * (1 - g) * lam);
    atomicAdd(L + (size_t)S.r0 * ld + S.c0 + 1, S.p0 * f * (1 - g) * lam);
    atomicAdd(L + (size_t)S.r1 * ld + S.c0, S.p1 * (1 - f) * g * lam);
    atomicAdd(L + (size_t)S.r1 * ld + S.c0 + 1, S.p1 * f * g * lam);
}

constexpr int MAX_ITER = 16;  // correctors the adjoint accepts

struct PAdjArgs {
    GridDev g;
    double dt;
    int n_iter;
    int ift;                  // 1: implicit-function theorem at the converged trapezoid
    double qm[4], qw[4];
    int massive[4];
    int64_t n;
    const double *x[5];       // state n: r, th, ur, ut, up
    const uint32_t *tag0;     // tags at n
    const uint32_t *tag1;     // tags at n+1
    const double *F[6];       // fields at n
    const double *tape;       // the forward push's record of step n (layout in grpic_internal.cuh)
    int64_t tape_ld;
    const double *lamJ[3];    // adjoint of J A
    const double *lam1[5];    // adjoint of state n+1
    double *lam0[5];          // adjoint of state n (output)
    double *lamF[6];          // adjoint of fields at n (accumulated)
    double *La;               // per particle: its part of dL/da (may be null)
    int64_t ld;
};

template <bool SPIN>
__global__ void __launch_bounds__(128) particle_adjoint(PAdjArgs A)
{
    constexpr int ND = SPIN ? 3 : 2;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.n) return;
    const GridDev &g = A.g;
    double out[5] = {0, 0, 0, 0, 0};
    uint32_t t0 = A.tag0[p];
    if (SPIN) A.La[p] = 0.0;
    if (t0 & DEAD) {
        for (int k = 0; k < 5; ++k) A.lam0[k][p] = 0.0;
        return;
    }
    const int sp = t0 & 3u;
    const bool massive = A.massive[sp] != 0, charged = massive && A.qm[sp] != 0.0;
    double r = A.x[0][p], th = A.x[1][p];
    double u[3] = {A.x[2][p], A.x[3][p], A.x[4][p]};
    // a state the push refused (outside the domain, non-finite) moved nothing
    bool inside = isfinite(r) && isfinite(th) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) &&
                  r >= g.r_in && r < g.r_out && th >= 0.0 && th <= M_PI;
    if (!inside) {
        for (int k = 0; k < 5; ++k) A.lam0[k][p] = 0.0;
        return;
    }
    double x1a = (log(r) - g.ln_rin) / g.dx1, x2a = th / g.dth;
    if (x1a >= (double)g.nr) x1a = nextafter((double)g.nr, 0.0);  // as in the push
    if (x1a < 0.0) x1a = 0.0;
    const double dt = A.dt, eps = massive ? 1.0 : 0.0;
    // the forward push's record: u' after the Boris step, the corrector
    // iterates, x^{n+1} before the reflection
    const double *T = A.tape + p;
    const int64_t tl = A.tape_ld;
    const int N = A.n_iter, te = tape_end(N);
    const double y0[5] = {r, th, T[(TAPE_U + 0) * tl], T[(TAPE_U + 1) * tl], T[(TAPE_U + 2) * tl]};
    const double s0 = T[TAPE_SC0 * tl], c0 = T[(TAPE_SC0 + 1) * tl];
    const double y1[5] = {T[te * tl], T[(te + 1) * tl], T[(te + 2) * tl], T[(te + 3) * tl], y0[4]};
    const double dphi = T[(te + 4) * tl];
    double refl = 1.0;
    double th1 = y1[1];
    if (th1 < 0.0) { th1 = -th1; refl = -1.0; }
    else if (th1 > M_PI) { th1 = 2.0 * M_PI - th1; refl = -1.0; }
    double x1b = (log(y1[0]) - g.ln_rin) / g.dx1, x2b = th1 / g.dth;
    int i0 = (int)floor(x1a), j0 = jcell(g, x2a);
    int di = (int)floor(x1b) - i0, dj = jcell(g, x2b) - j0;
    // the push's own checks: a finite end point, at most one cell away
    bool moved_ok = di >= -1 && di <= 1 && dj >= -1 && dj <= 1 && isfinite(x1b) && isfinite(x2b) &&
                    isfinite(y1[2]) && isfinite(y1[3]) && isfinite(dphi);
    if (!moved_ok) {
        for (int k = 0; k < 5; ++k) A.lam0[k][p] = 0.0;
        return;
    }

    // ---- adjoint -------------------------------------------------------
    double l1[5] = {0, 0, 0, 0, 0};
    if (!(A.tag1[p] & DEAD))
        for (int k = 0; k < 5; ++k) l1[k] = A.lam1[k][p];
    double ldphi = 0.0, lx1a = 0.0, lx2a = 0.0, lx1b = 0.0, lx2b = 0.0;
    double qw = A.qw[sp];
    if (qw != 0.0) {
        // transpose of the Esirkepov window (same algebra as the push), each
        // current's window contracted with its adjoint one row or column at a
        // time: J^r A_r(k+1/2, l) = cr P_r(k) (S1_t + S0_t)(l), J^th A_th
        // likewise, J^phi dV(k, l) = cq dphi (S1_r A_t + S0_r B_t)(k, l) with
        // A_t = S1_t / 3 + S0_t / 6, B_t = S1_t / 6 + S0_t / 3
        double S0r[4], S1r[4], S0t[4], S1t[4], dS0r[4], dS1r[4], dS0t[4], dS1t[4];
        for (int k = 0; k < 4; ++k) {
            double cr_ = i0 - 1 + k, ct = j0 - 1 + k;
            S0r[k] = W1(x1a - cr_); dS0r[k] = dW1(x1a - cr_);
            S1r[k] = W1(x1b - cr_); dS1r[k] = dW1(x1b - cr_);
            S0t[k] = W1(x2a - ct); dS0t[k] = dW1(x2a - ct);
            S1t[k] = W1(x2b - ct); dS1t[k] = dW1(x2b - ct);
        }
        const double cr = -qw / (2.0 * dt), cq = qw / dt, cp = cq * dphi;
        const double c3 = 1.0 / 3.0, c6 = 1.0 / 6.0;
        double Pr = 0.0, dPr1 = 0.0, dPr0 = 0.0;
        for (int k = 0; k < 3; ++k) {
            Pr += S1r[k] - S0r[k];
            dPr1 += dS1r[k];
            dPr0 += dS0r[k];
            double U = 0.0, V = 0.0, W = 0.0;
            for (int l = 0; l < 4; ++l) {
                int row = j0 - 1 + l;
                if (row < 0 || row > g.nth) continue;
                double L = A.lamJ[0][(size_t)row * A.ld + (i0 - 1 + k + NG)];
                U += L * (S1t[l] + S0t[l]);
                V += L * dS1t[l];
                W += L * dS0t[l];
            }
            lx1b += cr * dPr1 * U;
            lx1a -= cr * dPr0 * U;
            lx2b += cr * Pr * V;
            lx2a += cr * Pr * W;
        }
        double Pt = 0.0, dPt1 = 0.0, dPt0 = 0.0;
        for (int l = 0; l < 3; ++l) {
            Pt += S1t[l] - S0t[l];
            dPt1 += dS1t[l];
            dPt0 += dS0t[l];
            int row = j0 - 1 + l;
            if (row < 0 || row > g.nth - 1) continue;
            double U = 0.0, V = 0.0, W = 0.0;
            for (int k = 0; k < 4; ++k) {
                double L = A.lamJ[1][(size_t)row * A.ld + (i0 - 1 + k + NG)];
                U += L * (S1r[k] + S0r[k]);
                V += L * dS1r[k];
                W += L * dS0r[k];
            }
            lx1b += cr * Pt * V;
            lx1a += cr * Pt * W;
            lx2b += cr * dPt1 * U;
            lx2a -= cr * dPt0 * U;
        }
        double At[4], Bt[4], LC[4] = {0, 0, 0, 0}, LD[4] = {0, 0, 0, 0};
        for (int l = 0; l < 4; ++l) {
            At[l] = c3 * S1t[l] + c6 * S0t[l];
            Bt[l] = c6 * S1t[l] + c3 * S0t[l];
        }
        for (int k = 0; k < 4; ++k) {
            const double Ck = c3 * S1r[k] + c6 * S0r[k], Dk = c6 * S1r[k] + c3 * S0r[k];
            double LA = 0.0, LB = 0.0;
            for (int l = 0; l < 4; ++l) {
                int row = j0 - 1 + l;
                if (row < 0 || row > g.nth) continue;
                double L = A.lamJ[2][(size_t)row * A.ld + (i0 - 1 + k + NG)];
                LA += L * At[l];
                LB += L * Bt[l];
                LC[l] += L * Ck;
                LD[l] += L * Dk;
            }
            ldphi += cq * (S1r[k] * LA + S0r[k] * LB);
            lx1b += cp * dS1r[k] * LA;
            lx1a += cp * dS0r[k] * LB;
        }
        for (int l = 0; l < 4; ++l) {
            lx2b += cp * dS1t[l] * LC[l];
            lx2a += cp * dS0t[l] * LD[l];
        }
    }
    // end point: logical -> (r, theta) after reflection, then the reflection
    l1[0] += lx1b / (y1[0] * g.dx1);
    l1[1] += lx2b / g.dth;
    l1[1] *= refl;
    l1[3] *= refl;
    const double hh = 0.5 * dt;
    double l0[5];
    double la = 0.0;                       // dL/da through the metric of this push
    double *pla = &la;
    if (A.ift) {
        // the converged trapezoid y1 = y0 + dt/2 (F(y1) + F(y0)), dphi = dt/2
        // (X^ph(y1) + X^ph(y0)), by the implicit-function theorem:
        // (I - dt/2 dF/dy(y1))^T w = lambda_1, lambda_0 = (I + dt/2 dF/dy(y0))^T w
        double F1[5], J1[5][5], Fp1, dFp1[5];
        rhs_jac(g.a, eps, y1, F1, J1, Fp1, dFp1);
        for (int k = 0; k < 5; ++k) l1[k] += hh * ldphi * dFp1[k];
        double M[5][5];
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) M[a][b] = (a == b ? 1.0 : 0.0) - hh * J1[b][a];  // transposed
        double w[5] = {l1[0], l1[1], l1[2], l1[3], l1[4]};
        solve5(M, w);
        double hw[5], v0[5];
        for (int k = 0; k < 5; ++k) hw[k] = hh * w[k];
        if constexpr (SPIN) {
            // the a-dependence of F(y1): w . dt/2 dF/da(y1) + dt/2 ldphi dX^ph/da(y1)
            double unused[5], s1, c1;
            sincos(y1[1], &s1, &c1);
            rhs_vjp_p<ND>(g.a, eps, y1, s1, c1, hw, hh * ldphi, unused, pla);
        }
        rhs_vjp_p<ND>(g.a, eps, y0, s0, c0, hw, hh * ldphi, v0, pla);
        for (int k = 0; k < 5; ++k) l0[k] = w[k] + v0[k];
    } else {
        // transpose of the iteration the push runs: y~_0 = y0 + dt F(y0),
        // y~_{k+1} = y0 + dt/2 (F(y~_k) + F(y0)), dphi = dt/2 (X^ph(y~_{N-1}) + X^ph(y0))
        double gk[5] = {l1[0], l1[1], l1[2], l1[3], l1[4]};
        double lF0[5] = {0, 0, 0, 0, 0}, ly0[5] = {0, 0, 0, 0, 0}, lFp0 = 0.0;
        if (N == 0) {
            lFp0 += dt * ldphi;
        } else {
            for (int it = N - 1; it >= 0; --it) {
                for (int k = 0; k < 5; ++k) {
                    ly0[k] += gk[k];
                    lF0[k] += hh * gk[k];
                }
                double ap = (it == N - 1) ? hh * ldphi : 0.0;
                lFp0 += ap;
                double hg[5], gn[5];
                for (int k = 0; k < 5; ++k) hg[k] = hh * gk[k];
                const double *q = T + (int64_t)(TAPE_IT + 6 * it) * tl;
                const double yi[5] = {q[0], q[tl], q[2 * tl], q[3 * tl], y0[4]};
                rhs_vjp_p<ND>(g.a, eps, yi, q[4 * tl], q[5 * tl], hg, ap, gn, pla);
                for (int k = 0; k < 5; ++k) gk[k] = gn[k];
            }
        }
        for (int k = 0; k < 5; ++k) {
            ly0[k] += gk[k];
            lF0[k] += dt * gk[k];
        }
        double v0[5];
        rhs_vjp_p<ND>(g.a, eps, y0, s0, c0, lF0, lFp0, v0, pla);
        for (int k = 0; k < 5; ++k) l0[k] = ly0[k] + v0[k];
    }
    // start point: deposit's start-weight derivatives
    l0[0] += lx1a / (r * g.dx1);
    l0[1] += lx2a / g.dth;
    // Boris: y0 = (r, th, u'(r, th, u, E))
    out[0] = l0[0];
    out[1] = l0[1];
    if (charged) {
        // fields at x^n and their logical derivatives
        St S[6];
        double E[6], dE1[6], dE2[6];
        stencil(g, x1a, x2a, true, false, 1.0, S[0]);   // D^r
        stencil(g, x1a, x2a, false, true, -1.0, S[1]);  // D^th (odd across the axis)
        stencil(g, x1a, x2a, false, false, 1.0, S[2]);  // D^ph
        stencil(g, x1a, x2a, false, true, 1.0, S[3]);   // B^r
        stencil(g, x1a, x2a, true, false, 1.0, S[4]);   // B^th
        stencil(g, x1a, x2a, true, true, 1.0, S[5]);    // B^ph
        for (int c = 0; c < 6; ++c) gather_d(A.F[c], A.ld, S[c], E[c], dE1[c], dE2[c]);
        double zv[11] = {r, th, u[0], u[1], u[2], E[0], E[1], E[2], E[3], E[4], E[5]};
        double lb[11];
        boris_vjp<ND>(g.a, A.qm[sp], dt, zv, s0, c0, l0 + 2, lb, pla);
        out[0] += lb[0];
        out[1] += lb[1];
        for (int k = 0; k < 3; ++k) out[2 + k] = lb[2 + k];
        double lE[6];
        for (int c = 0; c < 6; ++c) lE[c] = lb[5 + c];
        double lx1 = 0.0, lx2 = 0.0;
        for (int c = 0; c < 6; ++c) {
            scatter_w(A.lamF[c], A.ld, S[c], lE[c]);
            lx1 += lE[c] * dE1[c];
            lx2 += lE[c] * dE2[c];
        }
        out[0] += lx1 / (r * g.dx1);
        out[1] += lx2 / g.dth;
    } else {
        for (int k = 0; k < 3; ++k) out[2 + k] = l0[2 + k];
    }
    for (int k = 0; k < 5; ++k) A.lam0[k][p] = out[k];
    if (SPIN) A.La[p] = la;
}

// ---- field update transpose -------------------------------------------------
struct FAdj {
    int nr, nth;
    int64_t ld, ldt;
    size_t slab;
    const double *tab, *col1d;
};

__device__ __forceinline__ double tb(const FAdj &A, int slot, int i, int j)
{
    return A.tab[slot * A.slab + (size_t)j * A.ldt + (i + NG)];
}

// lamC (6 arrays at physical points) -> aux adjoints lamA[0..5] = H_r, H_th,
// H_ph, E_r, E_th, E_ph (transpose of the circulations, Eqs. D-update, B-update)
__global__ void circ_T(FAdj A, const double *const *lamC, double *const *lamA, double dth)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > A.nr || j > A.nth) return;
    const int nr = A.nr, nth = A.nth;
    size_t q = (size_t)j * A.ld + (i + NG);
    auto at = [&](double *L, int ii, int jj, double v) { atomicAdd(L + (size_t)jj * A.ld + (ii + NG), v); };
    double drd = A.col1d[1 * A.ldt + i + NG], drp = A.col1d[0 * A.ldt + i + NG];
    if (i <= nr - 1) {
        double gv = lamC[0][q] * tb(A, T_INV_ADR, i, j);
        if (j < nth) at(lamA[2], i, j, gv);
        if (j > 0) at(lamA[2], i, j - 1, -gv);
    }
    if (j < nth) {
        double gv = lamC[1][q] * tb(A, T_INV_ADT, i, j);
        at(lamA[2], i - 1, j, gv);
        at(lamA[2], i, j, -gv);
        double gb = lamC[3][q] * tb(A, T_INV_ABR, i, j);
        at(lamA[5], i, j + 1, -gb);
        at(lamA[5], i, j, gb);
    }
    if (j > 0 && j < nth) {
        double gv = lamC[2][q] * tb(A, T_INV_ADP, i, j);
        at(lamA[1], i, j, gv * dth);
        at(lamA[1], i - 1, j, -gv * dth);
        at(lamA[0], i, j - 1, gv * drd);
        at(lamA[0], i, j, -gv * drd);
        if (i <= nr - 1) {
            double gb = lamC[4][q] * tb(A, T_INV_ABT, i, j);
            at(lamA[5], i, j, -gb);
            at(lamA[5], i + 1, j, gb);
        }
    }
    if (i <= nr - 1 && j < nth) {
        double gb = lamC[5][q] * tb(A, T_INV_ABP, i, j);
        at(lamA[4], i + 1, j, -gb * dth);
        at(lamA[4], i, j, gb * dth);
        at(lamA[3], i, j, -gb * drp);
        at(lamA[3], i, j + 1, gb * drp);
    }
}

// aux adjoints -> field adjoints (transpose of Eqs. auxH, auxE); one thread per
// storage column/row, scatter with atomics
__global__ void aux_T(FAdj A, const double *const *lamA, double *const *lamX)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (col < 1 || col > (int)A.ldt - 2 || j > A.nth) return;
    int i = col - NG;
    size_t q = (size_t)j * A.ld + col;
    auto at = [&](double *L, int ii, int jj, double v) {
        if (v != 0.0) atomicAdd(L + (size_t)jj * A.ld + (ii + NG), v);
    };
    double h;
    // fields: 0 D^r, 1 D^th, 2 D^ph, 3 B^r, 4 B^th, 5 B^ph
    if (j < A.nth) {
        h = lamA[0][q];  // H_r
        if (h != 0.0) {
            at(lamX[3], i, j, tb(A, T_AGRR_BR, i, j) * h);
            at(lamX[5], i, j, 0.5 * tb(A, T_AGRP_BP, i, j) * h);
            at(lamX[5], i - 1, j, 0.5 * tb(A, T_AGRP_BP, i - 1, j) * h);
        }
        h = lamA[2][q];  // H_ph
        if (h != 0.0) {
            at(lamX[5], i, j, tb(A, T_AGPP_BP, i, j) * h);
            at(lamX[3], i, j, 0.5 * tb(A, T_AGRP_BR, i, j) * h);
            at(lamX[3], i + 1, j, 0.5 * tb(A, T_AGRP_BR, i + 1, j) * h);
            at(lamX[1], i, j, -0.5 * tb(A, T_SGB_DT, i, j) * h);
            at(lamX[1], i + 1, j, -0.5 * tb(A, T_SGB_DT, i + 1, j) * h);
        }
        h = lamA[4][q];  // E_th
        if (h != 0.0) {
            at(lamX[1], i, j, tb(A, T_AGTT_DT, i, j) * h);
            at(lamX[5], i, j, -0.5 * tb(A, T_SGB_BP, i, j) * h);
            at(lamX[5], i - 1, j, -0.5 * tb(A, T_SGB_BP, i - 1, j) * h);
        }
    }
    h = lamA[1][q];  // H_th
    if (h != 0.0) {
        at(lamX[4], i, j, tb(A, T_AGTT_BT, i, j) * h);
        at(lamX[2], i, j, 0.5 * tb(A, T_SGB_DP, i, j) * h);
        at(lamX[2], i + 1, j, 0.5 * tb(A, T_SGB_DP, i + 1, j) * h);
    }
    h = lamA[3][q];  // E_r
    if (h != 0.0) {
        at(lamX[0], i, j, tb(A, T_AGRR_DR, i, j) * h);
        at(lamX[2], i, j, 0.5 * tb(A, T_AGRP_DP, i, j) * h);
        at(lamX[2], i + 1, j, 0.5 * tb(A, T_AGRP_DP, i + 1, j) * h);
    }
    h = lamA[5][q];  // E_ph
    if (h != 0.0) {
        at(lamX[2], i, j, tb(A, T_AGPP_DP, i, j) * h);
        at(lamX[0], i, j, 0.5 * tb(A, T_AGRP_DR, i, j) * h);
        at(lamX[0], i - 1, j, 0.5 * tb(A, T_AGRP_DR, i - 1, j) * h);
        at(lamX[4], i, j, 0.5 * tb(A, T_SGB_BT, i, j) * h);
        at(lamX[4], i - 1, j, 0.5 * tb(A, T_SGB_BT, i - 1, j) * h);
    }
}

__device__ __forceinline__ bool phys(int comp, int i, int j, int nr, int nth)
{
    bool half_r = (comp == 0 || comp == 4 || comp == 5), half_t = (comp == 1 || comp == 3 || comp == 5);
    if (i < 0 || i > (half_r ? nr - 1 : nr)) return false;
    if (j > (half_t ? nth - 1 : nth)) return false;
    return true;
}

// transpose of the boundary projection P of one stage (with damping when
// damp != 0): mu[phys] = damp * (lam[phys] + lam of the guard copies of it);
// axis D^ph, B^th rows and non-physical entries get 0
__global__ void proj_T(FAdj A, const double *const *lam, double *const *mu, int damp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > A.nr || j > A.nth) return;
    for (int comp = 0; comp < 6; ++comp) {
        size_t row = (size_t)j * A.ld;
        double v = 0.0;
        if (phys(comp, i, j, A.nr, A.nth) && !((comp == 2 || comp == 4) && (j == 0 || j == A.nth))) {
            bool half_r = (comp == 0 || comp == 4 || comp == 5);
            int last = half_r ? A.nr - 1 : A.nr;
            v = lam[comp][row + i + NG];
            if (i == 0) v += lam[comp][row + 0] + lam[comp][row + 1];
            if (i == last)
                for (int c = last + 1 + NG; c < A.nr + 2 * NG; ++c) v += lam[comp][row + c];
            if (damp) v *= A.col1d[(half_r ? 3 : 2) * A.ldt + i + NG];
        }
        mu[comp][row + i + NG] = v;
        if (i == 0) { mu[comp][row + 0] = 0.0; mu[comp][row + 1] = 0.0; }
        if (i == A.nr)
            for (int c = A.nr + 1 + NG; c < A.nr + 2 * NG; ++c) mu[comp][row + c] = 0.0;
    }
}

// entries a field update never writes (rows past the last half-theta row,
// columns past the last guard) keep their value: the identity
__global__ void passthru(FAdj A, const double *const *lamIn, double *const *lamOut)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (c >= A.ld || j > A.nth) return;
    size_t q = (size_t)j * A.ld + c;
    for (int comp = 0; comp < 6; ++comp) {
        bool half_t = (comp == 1 || comp == 3 || comp == 5);
        bool written = c < A.nr + 2 * NG && j <= (half_t ? A.nth - 1 : A.nth);
        if (!written) lamOut[comp][q] += lamIn[comp][q];
    }
}

// y[k] += s * x[k] over n elements of 6 arrays
__global__ void axpy6(double *const *y, const double *const *x, double s, size_t n)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    for (int k = 0; k < 6; ++k) y[k][e] += s * x[k][e];
}

// lamJ[k] (J A adjoint) += s * invA^D_k * mu_D[k] at physical D points
__global__ void jadj(FAdj A, const double *const *mu, double *const *lamJ, double s)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > A.nr || j > A.nth) return;
    const int inv[3] = {T_INV_ADR, T_INV_ADT, T_INV_ADP};
    for (int k = 0; k < 3; ++k)
        if (phys(k, i, j, A.nr, A.nth)) {
            size_t q = (size_t)j * A.ld + i + NG;
            lamJ[k][q] += s * tb(A, inv[k], i, j) * mu[k][q];
        }
}

// ---- objective ------------------------------------------------------------
__device__ __forceinline__ double fx(const double *F, int64_t ld, int i, int j) { return F[(size_t)j * ld + i + NG]; }

// auxiliary fields needed at the ring (same formulas as the field update)
struct Ring {
    double Eth, Hph, Eph, Hth;
};
__device__ Ring ring_vals(FAdj A, const double *const *F, int iH, int j)
{
    auto Hph = [&](int i, int jj) {
        return tb(A, T_AGPP_BP, i, jj) * fx(F[5], A.ld, i, jj) +
               0.5 * (tb(A, T_AGRP_BR, i, jj) * fx(F[3], A.ld, i, jj) + tb(A, T_AGRP_BR, i + 1, jj) * fx(F[3], A.ld, i + 1, jj)) -
               0.5 * (tb(A, T_SGB_DT, i, jj) * fx(F[1], A.ld, i, jj) + tb(A, T_SGB_DT, i + 1, jj) * fx(F[1], A.ld, i + 1, jj));
    };
    auto Hth = [&](int i, int jj) {
        return tb(A, T_AGTT_BT, i, jj) * fx(F[4], A.ld, i, jj) +
               0.5 * (tb(A, T_SGB_DP, i, jj) * fx(F[2], A.ld, i, jj) + tb(A, T_SGB_DP, i + 1, jj) * fx(F[2], A.ld, i + 1, jj));
    };
    auto Eth = [&](int i, int jj) {
        return tb(A, T_AGTT_DT, i, jj) * fx(F[1], A.ld, i, jj) -
               0.5 * (tb(A, T_SGB_BP, i, jj) * fx(F[5], A.ld, i, jj) + tb(A, T_SGB_BP, i - 1, jj) * fx(F[5], A.ld, i - 1, jj));
    };
    auto Eph = [&](int i, int jj) {
        return tb(A, T_AGPP_DP, i, jj) * fx(F[2], A.ld, i, jj) +
               0.5 * (tb(A, T_AGRP_DR, i, jj) * fx(F[0], A.ld, i, jj) + tb(A, T_AGRP_DR, i - 1, jj) * fx(F[0], A.ld, i - 1, jj)) +
               0.5 * (tb(A, T_SGB_BT, i, jj) * fx(F[4], A.ld, i, jj) + tb(A, T_SGB_BT, i - 1, jj) * fx(F[4], A.ld, i - 1, jj));
    };
    Ring R;
    R.Eth = Eth(iH, j);
    R.Hph = 0.5 * (Hph(iH - 1, j) + Hph(iH, j));
    R.Eph = 0.5 * (Eph(iH, j) + Eph(iH, j + 1));
    R.Hth = 0.25 * (Hth(iH - 1, j) + Hth(iH, j) + Hth(iH - 1, j + 1) + Hth(iH, j + 1));
    return R;
}

// flux at the ring (one block reduction) accumulated into *out with weight w
__global__ void flux_kernel(FAdj A, const double *const *F, int iH, double dth, double w, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int j = threadIdx.x; j < A.nth; j += blockDim.x) {
        Ring R = ring_vals(A, F, iH, j);
        s += (R.Eth * R.Hph - R.Eph * R.Hth) * dth;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out += w * red[0];
}

// seed: aux adjoints of w * flux (then aux_T maps them to the fields)
__global__ void flux_seed(FAdj A, const double *const *F, int iH, double dth, double w, double *const *lamA)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.nth) return;
    Ring R = ring_vals(A, F, iH, j);
    double c = w * dth;
    auto at = [&](int comp, int i, int jj, double v) { atomicAdd(lamA[comp] + (size_t)jj * A.ld + i + NG, v); };
    // aux order: 0 H_r, 1 H_th, 2 H_ph, 3 E_r, 4 E_th, 5 E_ph
    at(4, iH, j, c * R.Hph);
    at(2, iH - 1, j, 0.5 * c * R.Eth);
    at(2, iH, j, 0.5 * c * R.Eth);
    at(5, iH, j, -0.5 * c * R.Hth);
    at(5, iH, j + 1, -0.5 * c * R.Hth);
    for (int di = -1; di <= 0; ++di)
        for (int dj = 0; dj <= 1; ++dj) at(1, iH + di, j + dj, -0.25 * c * R.Eph);
}

// ---- spin derivative of the field update and of the objective -------------
// At fixed fields the update and the flux depend on the spin only through
// the static tables (face-area inverses, metric products of the auxiliary
// fields); dtab holds their a-derivatives.  A value and its a-derivative:
struct VD {
    double v, d;
};
__device__ __forceinline__ VD operator+(VD x, VD y) { return {x.v + y.v, x.d + y.d}; }
__device__ __forceinline__ VD operator-(VD x, VD y) { return {x.v - y.v, x.d - y.d}; }
__device__ __forceinline__ VD operator*(double c, VD x) { return {c * x.v, c * x.d}; }

// auxiliary fields of App. B (the field update's formulas) with their
// a-derivatives at fixed X
struct DAux {
    FAdj A;
    const double *dtab;
    const double *const *X;
    __device__ VD p(int slot, int comp, int i, int j) const
    {
        size_t q = slot * A.slab + (size_t)j * A.ldt + (i + NG);
        double x = X[comp][(size_t)j * A.ld + (i + NG)];
        return {A.tab[q] * x, dtab[q] * x};
    }
    __device__ VD t(int slot, int i, int j) const
    {
        size_t q = slot * A.slab + (size_t)j * A.ldt + (i + NG);
        return {A.tab[q], dtab[q]};
    }
    __device__ VD Hr(int i, int j) const
    {
        return p(T_AGRR_BR, 3, i, j) + 0.5 * (p(T_AGRP_BP, 5, i, j) + p(T_AGRP_BP, 5, i - 1, j));
    }
    __device__ VD Hth(int i, int j) const
    {
        return p(T_AGTT_BT, 4, i, j) + 0.5 * (p(T_SGB_DP, 2, i, j) + p(T_SGB_DP, 2, i + 1, j));
    }
    __device__ VD Hph(int i, int j) const
    {
        return p(T_AGPP_BP, 5, i, j) + 0.5 * (p(T_AGRP_BR, 3, i, j) + p(T_AGRP_BR, 3, i + 1, j)) -
               0.5 * (p(T_SGB_DT, 1, i, j) + p(T_SGB_DT, 1, i + 1, j));
    }
    __device__ VD Er(int i, int j) const
    {
        return p(T_AGRR_DR, 0, i, j) + 0.5 * (p(T_AGRP_DP, 2, i, j) + p(T_AGRP_DP, 2, i + 1, j));
    }
    __device__ VD Eth(int i, int j) const
    {
        return p(T_AGTT_DT, 1, i, j) - 0.5 * (p(T_SGB_BP, 5, i, j) + p(T_SGB_BP, 5, i - 1, j));
    }
    __device__ VD Eph(int i, int j) const
    {
        return p(T_AGPP_DP, 2, i, j) + 0.5 * (p(T_AGRP_DR, 0, i, j) + p(T_AGRP_DR, 0, i - 1, j)) +
               0.5 * (p(T_SGB_BT, 4, i, j) + p(T_SGB_BT, 4, i - 1, j));
    }
};

// block sum of v added to *out (blockDim.x * blockDim.y = 256)
__device__ __forceinline__ void block_add(double v, double *out)
{
    __shared__ double red[256];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0 && red[0] != 0.0) atomicAdd(out, red[0]);
}

// *out += sum over points of w . dC/da (X): C the circulation of one stage
// (Eqs. D-update, B-update divided by the face areas), w adjoint-shaped
__global__ void __launch_bounds__(256) dcirc_dot(FAdj A, const double *dtab, const double *const *X,
                                                 const double *const *w, double dth, double *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    double acc = 0.0;
    if (i <= A.nr && j <= A.nth) {
        DAux X_{A, dtab, X};
        const int nr = A.nr, nth = A.nth;
        const size_t q = (size_t)j * A.ld + (i + NG);
        const double drd = A.col1d[1 * A.ldt + i + NG], drp = A.col1d[0 * A.ldt + i + NG];
        auto term = [&](int comp, int inv_slot, VD circ) {
            VD inv = X_.t(inv_slot, i, j);
            return w[comp][q] * (circ.d * inv.v + circ.v * inv.d);
        };
        if (i <= nr - 1) {
            VD hp = (j < nth) ? X_.Hph(i, j) : VD{0.0, 0.0};
            VD hm = (j > 0) ? X_.Hph(i, j - 1) : VD{0.0, 0.0};
            acc += term(0, T_INV_ADR, hp - hm);
        }
        if (j < nth) {
            acc += term(1, T_INV_ADT, X_.Hph(i - 1, j) - X_.Hph(i, j));
            acc += term(3, T_INV_ABR, -1.0 * (X_.Eph(i, j + 1) - X_.Eph(i, j)));
        }
        if (j > 0 && j < nth) {
            acc += term(2, T_INV_ADP, dth * (X_.Hth(i, j) - X_.Hth(i - 1, j)) + drd * (X_.Hr(i, j - 1) - X_.Hr(i, j)));
            if (i <= nr - 1) acc += term(4, T_INV_ABT, -1.0 * (X_.Eph(i, j) - X_.Eph(i + 1, j)));
        }
        if (i <= nr - 1 && j < nth)
            acc += term(5, T_INV_ABP,
                        -1.0 * (dth * (X_.Eth(i + 1, j) - X_.Eth(i, j)) + drp * (X_.Er(i, j) - X_.Er(i, j + 1))));
    }
    block_add(acc, out);
}

// *out += sj * sum over the D points a stage writes of w . d(invA)/da J A
// (the current term of Eq. fld-predictor / fld-corrector)
__global__ void __launch_bounds__(256) jinv_dot(FAdj A, const double *dtab, const double *const *w,
                                                const double *const *J, double sj, double *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    double acc = 0.0;
    if (i <= A.nr && j <= A.nth) {
        const size_t q = (size_t)j * A.ld + (i + NG), qt = (size_t)j * A.ldt + (i + NG);
        if (i <= A.nr - 1) acc += w[0][q] * dtab[T_INV_ADR * A.slab + qt] * J[0][q];
        if (j < A.nth) acc += w[1][q] * dtab[T_INV_ADT * A.slab + qt] * J[1][q];
        if (j > 0 && j < A.nth) acc += w[2][q] * dtab[T_INV_ADP * A.slab + qt] * J[2][q];
    }
    block_add(sj * acc, out);
}

// *out += w * d(flux)/da at fixed fields F (the ring values of the objective)
__global__ void __launch_bounds__(256) flux_da(FAdj A, const double *dtab, const double *const *F, int iH, double dth,
                                               double w, double *out)
{
    double acc = 0.0;
    int j = blockIdx.x * 256 + threadIdx.x;
    if (j < A.nth) {
        DAux X_{A, dtab, F};
        VD Eth = X_.Eth(iH, j);
        VD Hph = 0.5 * (X_.Hph(iH - 1, j) + X_.Hph(iH, j));
        VD Eph = 0.5 * (X_.Eph(iH, j) + X_.Eph(iH, j + 1));
        VD Hth = 0.25 * (X_.Hth(iH - 1, j) + X_.Hth(iH, j) + X_.Hth(iH - 1, j + 1) + X_.Hth(iH, j + 1));
        acc = w * dth * (Eth.d * Hph.v + Eth.v * Hph.d - Eph.d * Hth.v - Eph.v * Hth.d);
    }
    block_add(acc, out);
}

// dtab = (tab(a + h) - tab(a - h)) / (2h)
__global__ void central_diff(const double *tp, const double *tm, double inv2h, size_t n, double *d)
{
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) d[e] = (tp[e] - tm[e]) * inv2h;
}

// *out += sum of x[0..n)
__global__ void __launch_bounds__(256) sum_into(const double *x, int64_t n, double *out)
{
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) acc += x[e];
    block_add(acc, out);
}

}  // namespace
}  // namespace grpic

using namespace grpic;

namespace {

struct Bufs {
    size_t fn;      // elements of one field array
    int64_t np;     // particles
};

// device pointer arrays for kernels taking "double *const *" (6 entries)
struct PtrSet {
    double **d;  // device array of 6 (or 3) pointers
};

cudaError_t upload_ptrs(double *const *h, int n, double ***d, cudaStream_t s)
{
    cudaError_t e = cudaMalloc(d, sizeof(double *) * n);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*d, h, sizeof(double *) * n, cudaMemcpyHostToDevice, s);
}

}  // namespace

extern "C" grpic_status grpic_horizon_flux(grpic_ctx *ctx, const grpic_fields *f, int i_horizon, double *out,
                                           void *stream)
{
    if (!ctx || !f || !out || ctx->prm.precision != 64 || f->ld < ctx->g.nr + 2 * NG || i_horizon < 1 ||
        i_horizon > ctx->g.nr - 1)
        return GRPIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *hp[6];
    for (int k = 0; k < 3; ++k) {
        hp[k] = (double *)f->D[k];
        hp[3 + k] = (double *)f->B[k];
    }
    double **dp = nullptr;
    if (upload_ptrs(hp, 6, &dp, s) != cudaSuccess) return GRPIC_ENOMEM;
    FAdj A{ctx->g.nr, ctx->g.nth, f->ld, ctx->g.ld_tab, ctx->slab, ctx->tab, ctx->col1d};
    cudaMemsetAsync(out, 0, sizeof(double), s);
    flux_kernel<<<1, 256, 0, s>>>(A, dp, i_horizon, ctx->g.dth, 1.0, out);
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(s);
    cudaFree(dp);
    return e == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}

// What the spin derivative of one field update needs: the derivative
// tables, the update's input fields Xn, its currents J and every stage's
// output Y[k] (device pointer arrays), and the scalar it accumulates into.
struct SpinField {
    const double *dtab;
    double **Xn;   // 6
    double **J;    // 3
    double **Y;    // (n_field_iter + 1) * 6
    double *La;
};

// Transpose of one field update: lam (adjoint of F^{n+1}, in f_lam->D/B) ->
// adjoint of F^n (out->D/B) and of the integrated currents J A (out->J).
// With sp, also adds the update's a-derivative contracted with the stage
// adjoints to sp->La: every stage's pre-projection value
//   dt (c_k C(Xn) + beta_s C(Y_{k-1})) - dt invA J   (c_0 = 1, c_k = alpha_s)
// depends on a through the tables of C and invA.
static grpic_status field_adjoint(grpic_ctx *ctx, double **lamIn, double **lamOut, double **lamJ, double **work,
                                  int64_t ld, cudaStream_t s, double ***dptrs, const SpinField *sp = nullptr)
{
    // work: mu[6], lamCn[6], lamPrev[6], aux[6]  (24 arrays); dptrs: device copies
    const int N = ctx->prm.n_field_iter;
    const double dt = ctx->prm.dt, bs = ctx->prm.beta_field, as = 1.0 - bs;
    size_t fn = (size_t)(ctx->g.nth + 1) * ld;
    FAdj A{ctx->g.nr, ctx->g.nth, ld, ctx->g.ld_tab, ctx->slab, ctx->tab, ctx->col1d};
    dim3 blk(64, 4), grd((ctx->g.nr + 1 + 63) / 64, (ctx->g.nth + 1 + 3) / 4);
    dim3 gfull((ctx->g.ld_tab + 63) / 64, (ctx->g.nth + 1 + 3) / 4);
    unsigned nb = (unsigned)((fn + 255) / 256);
    double **d_in = dptrs[0], **d_out = dptrs[1], **d_J = dptrs[2], **d_mu = dptrs[3], **d_lcn = dptrs[4],
           **d_prev = dptrs[5], **d_aux = dptrs[6], **d_cur = dptrs[7];
    double **mu = work, **lcn = work + 6, **prev = work + 12, **aux = work + 18;
    for (int k = 0; k < 6; ++k) {
        cudaMemsetAsync(lamOut[k], 0, fn * sizeof(double), s);
        cudaMemsetAsync(lcn[k], 0, fn * sizeof(double), s);
        cudaMemsetAsync(mu[k], 0, fn * sizeof(double), s);
    }
    for (int k = 0; k < 3; ++k) cudaMemsetAsync(lamJ[k], 0, fn * sizeof(double), s);
    dim3 gld((unsigned)((ld + 63) / 64), (ctx->g.nth + 1 + 3) / 4);
    passthru<<<gld, blk, 0, s>>>(A, d_in, d_out);
    // current adjoint of the stage output: starts at lamIn
    cudaMemcpyAsync(d_cur, d_in, sizeof(double *) * 6, cudaMemcpyDeviceToDevice, s);
    for (int k = N; k >= 0; --k) {
        // mu = P_k^T lam_k (damping in the last stage)
        proj_T<<<grd, blk, 0, s>>>(A, d_cur, d_mu, (k == N && N > 0) ? 1 : 0);
        // lam X^n (physical part) += mu; lam Cn += dt * (k==0 ? 1 : alpha) * mu; lam J -= dt * invA * mu
        axpy6<<<nb, 256, 0, s>>>(d_out, d_mu, 1.0, fn);
        axpy6<<<nb, 256, 0, s>>>(d_lcn, d_mu, dt * (k == 0 ? 1.0 : as), fn);
        jadj<<<grd, blk, 0, s>>>(A, d_mu, d_J, -dt);
        if (sp)  // the current term: -dt mu_k . d(invA)/da J
            jinv_dot<<<grd, blk, 0, s>>>(A, sp->dtab, d_mu, sp->J, -dt, sp->La);
        if (k > 0) {
            // lam of the previous iterate = C^T (dt beta mu)
            for (int c = 0; c < 6; ++c) {
                cudaMemsetAsync(aux[c], 0, fn * sizeof(double), s);
                cudaMemsetAsync(prev[c], 0, fn * sizeof(double), s);
            }
            // scale mu by dt*beta in place
            axpy6<<<nb, 256, 0, s>>>(d_mu, d_mu, dt * bs - 1.0, fn);
            if (sp)  // dt beta_s mu_k . dC/da (Y_{k-1})
                dcirc_dot<<<grd, blk, 0, s>>>(A, sp->dtab, sp->Y + (k - 1) * 6, d_mu, ctx->g.dth, sp->La);
            circ_T<<<grd, blk, 0, s>>>(A, d_mu, d_aux, ctx->g.dth);
            aux_T<<<gfull, blk, 0, s>>>(A, d_aux, d_prev);
            cudaMemcpyAsync(d_cur, d_prev, sizeof(double *) * 6, cudaMemcpyDeviceToDevice, s);
        }
    }
    // (sum_k dt c_k mu_k) . dC/da (X^n)
    if (sp) dcirc_dot<<<grd, blk, 0, s>>>(A, sp->dtab, sp->Xn, d_lcn, ctx->g.dth, sp->La);
    // lam X^n += C^T lam Cn
    for (int c = 0; c < 6; ++c) cudaMemsetAsync(aux[c], 0, fn * sizeof(double), s);
    circ_T<<<grd, blk, 0, s>>>(A, d_lcn, d_aux, ctx->g.dth);
    aux_T<<<gfull, blk, 0, s>>>(A, d_aux, d_out);
    (void)lamIn;
    return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}

extern "C" grpic_status grpic_adjoint_field_step(grpic_ctx *ctx, const grpic_fields *lam_in, grpic_fields *lam_out,
                                                 void *stream)
{
    if (!ctx || !lam_in || !lam_out || ctx->prm.precision != 64 || lam_in->ld != lam_out->ld ||
        lam_in->ld < ctx->g.nr + 2 * NG || ctx->prm.n_field_iter < 1)
        return GRPIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t ld = lam_in->ld;
    size_t fn = (size_t)(ctx->g.nth + 1) * ld;
    std::vector<double *> work(24, nullptr);
    for (auto &w : work)
        if (cudaMalloc(&w, fn * sizeof(double)) != cudaSuccess) return GRPIC_ENOMEM;
    double *in[6], *out[6], *J[3];
    for (int k = 0; k < 3; ++k) {
        in[k] = (double *)lam_in->D[k];
        in[3 + k] = (double *)lam_in->B[k];
        out[k] = (double *)lam_out->D[k];
        out[3 + k] = (double *)lam_out->B[k];
        J[k] = (double *)lam_out->J[k];
    }
    double **dp[8];
    double *cur_dummy[6] = {0};
    bool ok = upload_ptrs(in, 6, &dp[0], s) == cudaSuccess && upload_ptrs(out, 6, &dp[1], s) == cudaSuccess &&
              upload_ptrs(J, 3, &dp[2], s) == cudaSuccess && upload_ptrs(&work[0], 6, &dp[3], s) == cudaSuccess &&
              upload_ptrs(&work[6], 6, &dp[4], s) == cudaSuccess && upload_ptrs(&work[12], 6, &dp[5], s) == cudaSuccess &&
              upload_ptrs(&work[18], 6, &dp[6], s) == cudaSuccess && upload_ptrs(cur_dummy, 6, &dp[7], s) == cudaSuccess;
    grpic_status st = ok ? field_adjoint(ctx, in, out, J, work.data(), ld, s, dp) : GRPIC_ENOMEM;
    cudaStreamSynchronize(s);
    for (int k = 0; k < 8; ++k)
        if (ok) cudaFree(dp[k]);
    for (auto w : work) cudaFree(w);
    return st;
}

// ---------------------------------------------------------------------------
// full gradient: forward with checkpoints, reverse sweep
// ---------------------------------------------------------------------------
extern "C" grpic_status grpic_adjoint_grad(grpic_ctx *ctx, const grpic_particles *p0, const grpic_fields *f0,
                                           int nsteps, int checkpoint_every, int i_horizon, int trapezoid_ift,
                                           double *L_out, double *const grad_p[5], double *const grad_f[6],
                                           double *dL_da, void *stream)
{
    if (!ctx || !p0 || !f0 || !L_out || ctx->prm.precision != 64 || nsteps < 1 || checkpoint_every < 1 ||
        i_horizon < 1 || i_horizon > ctx->g.nr - 1 || ctx->prm.n_field_iter < 1 || f0->ld < ctx->g.nr + 2 * NG ||
        p0->n < 0 || p0->n > INT32_MAX || (!grad_p && (grad_f || dL_da)) || ctx->prm.n_push_iter > MAX_ITER ||
        ctx->prm.pusher != 0 || ctx->prm.shape_order != 1 || ctx->prm.radiation != 0 || ctx->prm.injection != 0)
        return GRPIC_EINVAL;
    const bool want = grad_p != nullptr;  // NULL: the objective alone
    if (want)
        for (int k = 0; k < 5; ++k)
            if (!grad_p[k]) return GRPIC_EINVAL;
    if (p0->n > 0 && (!p0->x1 || !p0->x2 || !p0->u1 || !p0->u2 || !p0->u3 || !p0->tag)) return GRPIC_EINVAL;
    for (int k = 0; k < 3; ++k)
        if (!f0->D[k] || !f0->B[k]) return GRPIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ld = f0->ld, np = p0->n;
    const size_t fn = (size_t)(ctx->g.nth + 1) * ld;
    const int ck = checkpoint_every;
    const int nseg = (nsteps + ck - 1) / ck;
    std::vector<void *> allocs;
    auto dalloc = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, bytes > 0 ? bytes : 8) != cudaSuccess) return nullptr;
        allocs.push_back(q);
        return q;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        for (void *q : allocs) cudaFree(q);
    };
    // states: checkpoints (nseg) and the current segment's states (ck + 1)
    struct State {
        double *F[6];
        double *x[5];
        uint32_t *tag;
    };
    auto new_state = [&](State &S) -> bool {
        for (int k = 0; k < 6; ++k)
            if (!(S.F[k] = (double *)dalloc(fn * sizeof(double)))) return false;
        for (int k = 0; k < 5; ++k)
            if (!(S.x[k] = (double *)dalloc(np * sizeof(double)))) return false;
        return (S.tag = (uint32_t *)dalloc(np * sizeof(uint32_t))) != nullptr;
    };
    std::vector<State> cks(want ? nseg : 0), seg(want ? ck + 1 : 0);
    bool ok = true;
    for (auto &S : cks) ok = ok && new_state(S);
    for (auto &S : seg) ok = ok && new_state(S);
    // working particles / fields for the forward runs
    State W;
    ok = ok && new_state(W);
    double *Jw[3];
    for (int k = 0; k < 3; ++k) ok = ok && (Jw[k] = (double *)dalloc(fn * sizeof(double)));
    int64_t *cnt = (int64_t *)dalloc(sizeof(int64_t));
    double *Ldev = (double *)dalloc(sizeof(double));
    // adjoint arrays
    double *lamF[6], *lamF2[6], *lamJ[3], *lamP[5], *lamP2[5], *aux[6];
    for (int k = 0; k < 6; ++k) {
        ok = ok && (lamF[k] = (double *)dalloc(fn * sizeof(double)));
        ok = ok && (lamF2[k] = (double *)dalloc(fn * sizeof(double)));
        ok = ok && (aux[k] = (double *)dalloc(fn * sizeof(double)));
    }
    for (int k = 0; k < 3; ++k) ok = ok && (lamJ[k] = (double *)dalloc(fn * sizeof(double)));
    for (int k = 0; k < 5; ++k) {
        ok = ok && (lamP[k] = (double *)dalloc(np * sizeof(double)));
        ok = ok && (lamP2[k] = (double *)dalloc(np * sizeof(double)));
    }
    // the forward push's record of every step of the current segment
    const int TW = tape_width(ctx->prm.n_push_iter);
    double *tape = want ? (double *)dalloc((size_t)ck * TW * (size_t)np * sizeof(double)) : nullptr;
    ok = ok && (!want || tape);
    std::vector<double *> work(want ? 24 : 0, nullptr);
    for (auto &w : work) ok = ok && (w = (double *)dalloc(fn * sizeof(double)));
    // spin derivative: derivative tables, per-particle parts, the segment's
    // currents and one update's stage outputs
    const bool spin = dL_da != nullptr;
    const int NF = ctx->prm.n_field_iter;
    const size_t ntab = ctx->slab * T_COUNT;
    double *dtab = nullptr, *Ladev = nullptr, *Lap = nullptr;
    std::vector<double *> segJ(spin ? 3 * ck : 0, nullptr), Ystage(spin ? 6 * (NF + 1) : 0, nullptr);
    if (spin) {
        ok = ok && (dtab = (double *)dalloc(ntab * sizeof(double)));
        ok = ok && (Ladev = (double *)dalloc(sizeof(double)));
        ok = ok && (Lap = (double *)dalloc(np * sizeof(double)));
        for (auto &q : segJ) ok = ok && (q = (double *)dalloc(fn * sizeof(double)));
        for (auto &q : Ystage) ok = ok && (q = (double *)dalloc(fn * sizeof(double)));
    }
    if (!ok) {
        cleanup();
        return GRPIC_ENOMEM;
    }
    if (spin) {
        // a-derivatives of the tables by central differences, h = 1e-5 (the
        // quadratures are smooth in a: truncation ~h^2, rounding ~1e-16/h)
        const double h = 1e-5;
        double *tp = (double *)dalloc(ntab * sizeof(double)), *tm = (double *)dalloc(ntab * sizeof(double));
        double *c1 = (double *)dalloc(4 * ctx->g.ld_tab * sizeof(double));
        if (!tp || !tm || !c1 || launch_tables_at(ctx, ctx->g.a + h, tp, c1, s) != cudaSuccess ||
            launch_tables_at(ctx, ctx->g.a - h, tm, c1, s) != cudaSuccess) {
            cleanup();
            return GRPIC_ENOMEM;
        }
        central_diff<<<(unsigned)((ntab + 255) / 256), 256, 0, s>>>(tp, tm, 0.5 / h, ntab, dtab);
        cudaMemsetAsync(Ladev, 0, sizeof(double), s);
    }
    auto copy_state = [&](State &dst, const State &src) {
        for (int k = 0; k < 6; ++k) cudaMemcpyAsync(dst.F[k], src.F[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
        for (int k = 0; k < 5; ++k) cudaMemcpyAsync(dst.x[k], src.x[k], np * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(dst.tag, src.tag, np * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    };
    // initial state -> W
    for (int k = 0; k < 3; ++k) {
        cudaMemcpyAsync(W.F[k], f0->D[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(W.F[3 + k], f0->B[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
    void *px[5] = {p0->x1, p0->x2, p0->u1, p0->u2, p0->u3};
    for (int k = 0; k < 5; ++k) cudaMemcpyAsync(W.x[k], px[k], np * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(W.tag, p0->tag, np * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(cnt, &np, sizeof(int64_t), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(Ldev, 0, sizeof(double), s);

    grpic_fields FW;
    for (int k = 0; k < 3; ++k) {
        FW.D[k] = W.F[k];
        FW.B[k] = W.F[3 + k];
        FW.J[k] = Jw[k];
    }
    FW.ld = ld;
    grpic_particles PW;
    memset(&PW, 0, sizeof PW);
    PW.n = np;
    PW.capacity = np;
    PW.d_count = nullptr;
    PW.x1 = W.x[0];
    PW.x2 = W.x[1];
    PW.u1 = W.x[2];
    PW.u2 = W.x[3];
    PW.u3 = W.x[4];
    PW.tag = W.tag;
    double *Wf[6];
    for (int k = 0; k < 6; ++k) Wf[k] = W.F[k];
    double **dWf = nullptr, **dLamF = nullptr, **dLamF2 = nullptr, **dAux = nullptr, **dSegF = nullptr;
    ok = upload_ptrs(Wf, 6, &dWf, s) == cudaSuccess && upload_ptrs(lamF, 6, &dLamF, s) == cudaSuccess &&
         upload_ptrs(lamF2, 6, &dLamF2, s) == cudaSuccess && upload_ptrs(aux, 6, &dAux, s) == cudaSuccess &&
         cudaMalloc(&dSegF, sizeof(double *) * 6) == cudaSuccess;
    if (ok) {
        allocs.push_back(dWf);
        allocs.push_back(dLamF);
        allocs.push_back(dLamF2);
        allocs.push_back(dAux);
        allocs.push_back(dSegF);
    } else {
        cleanup();
        return GRPIC_ENOMEM;
    }
    FAdj A{ctx->g.nr, ctx->g.nth, ld, ctx->g.ld_tab, ctx->slab, ctx->tab, ctx->col1d};
    const double wL = 1.0 / nsteps, dth = ctx->g.dth;
    grpic_status st = GRPIC_OK;
    // one forward step; with a tape slice, the push also records itself there
    auto fwd_step = [&](double *tp) -> grpic_status {
        for (int k = 0; k < 3; ++k) cudaMemsetAsync(Jw[k], 0, fn * sizeof(double), s);
        cudaError_t e = tp ? launch_push64_tape(ctx, &PW, &FW, tp, np, s)
                           : launch_push64(ctx, &PW, &PW, nullptr, nullptr, nullptr, &FW, false, s);
        if (e != cudaSuccess) return GRPIC_ECUDA;
        grpic_status r = GRPIC_OK;
        if (launch_field64(ctx, &FW, s) != cudaSuccess) r = GRPIC_ECUDA;
        return r;
    };
    // ---- forward with checkpoints --------------------------------------
    if (ensure_field_scratch_ext(ctx, ld) != GRPIC_OK || ensure_particle_scratch_ext(ctx, np) != GRPIC_OK) {
        cleanup();
        return GRPIC_ENOMEM;
    }
    // the last segment, the first the reverse sweep needs, is recorded here
    // (its states, the push's record and, for the spin derivative, its
    // currents) instead of being recomputed from its checkpoint
    const int last0 = (nseg - 1) * ck;
    for (int n = 0; n < nsteps && st == GRPIC_OK; ++n) {
        if (want && n % ck == 0) copy_state(cks[n / ck], W);
        const bool rec = want && n >= last0;
        const int m = n - last0;
        if (rec && m == 0) copy_state(seg[0], W);
        st = fwd_step(rec ? tape + (size_t)m * TW * (size_t)np : nullptr);
        if (rec) {
            copy_state(seg[m + 1], W);
            if (spin)
                for (int k = 0; k < 3; ++k)
                    cudaMemcpyAsync(segJ[3 * m + k], Jw[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
        flux_kernel<<<1, 256, 0, s>>>(A, dWf, i_horizon, dth, wL, Ldev);
        if (spin)  // the objective's own tables at F^{n+1}
            flux_da<<<(ctx->g.nth + 255) / 256, 256, 0, s>>>(A, dtab, dWf, i_horizon, dth, wL, Ladev);
    }
    cudaMemcpyAsync(L_out, Ldev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!want) {
        int hst = 0;
        cudaMemcpyAsync(&hst, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
        ctx->keys_valid = 0;
        ctx->hist_valid = 0;
        cleanup();
        if (cudaGetLastError() != cudaSuccess && st == GRPIC_OK) st = GRPIC_ECUDA;
        if (st == GRPIC_OK && hst != 0) st = (grpic_status)hst;
        return st;
    }
    // ---- reverse sweep -----------------------------------------------------
    for (int k = 0; k < 6; ++k) cudaMemsetAsync(lamF[k], 0, fn * sizeof(double), s);
    for (int k = 0; k < 5; ++k) cudaMemsetAsync(lamP[k], 0, np * sizeof(double), s);
    double **dptrs[8];
    double *Jl[3] = {lamJ[0], lamJ[1], lamJ[2]};
    double *cur_dummy[6] = {0};
    ok = upload_ptrs(lamF, 6, &dptrs[0], s) == cudaSuccess && upload_ptrs(lamF2, 6, &dptrs[1], s) == cudaSuccess &&
         upload_ptrs(Jl, 3, &dptrs[2], s) == cudaSuccess && upload_ptrs(&work[0], 6, &dptrs[3], s) == cudaSuccess &&
         upload_ptrs(&work[6], 6, &dptrs[4], s) == cudaSuccess && upload_ptrs(&work[12], 6, &dptrs[5], s) == cudaSuccess &&
         upload_ptrs(&work[18], 6, &dptrs[6], s) == cudaSuccess && upload_ptrs(cur_dummy, 6, &dptrs[7], s) == cudaSuccess;
    if (!ok) {
        cleanup();
        return GRPIC_ENOMEM;
    }
    for (int k = 0; k < 8; ++k) allocs.push_back(dptrs[k]);
    SpinField spf{dtab, nullptr, nullptr, nullptr, Ladev};
    if (spin) {
        ok = upload_ptrs(Ystage.data(), 6 * (NF + 1), &spf.Y, s) == cudaSuccess;
        if (ok) allocs.push_back(spf.Y);
        ok = ok && cudaMalloc(&spf.Xn, sizeof(double *) * 6) == cudaSuccess;
        if (ok) allocs.push_back(spf.Xn);
        ok = ok && cudaMalloc(&spf.J, sizeof(double *) * 3) == cudaSuccess;
        if (ok) allocs.push_back(spf.J);
        if (!ok) {
            cleanup();
            return GRPIC_ENOMEM;
        }
    }
    dim3 gfull((ctx->g.ld_tab + 63) / 64, (ctx->g.nth + 1 + 3) / 4), blk(64, 4);
    for (int sgi = nseg - 1; sgi >= 0 && st == GRPIC_OK; --sgi) {
        int n0 = sgi * ck, len = std::min(ck, nsteps - n0);
        // recompute the segment's states (the last one was recorded in the forward pass)
        if (sgi != nseg - 1) {
            copy_state(W, cks[sgi]);
            copy_state(seg[0], W);
        }
        for (int m = 0; m < len && st == GRPIC_OK && sgi != nseg - 1; ++m) {
            st = fwd_step(tape + (size_t)m * TW * (size_t)np);
            copy_state(seg[m + 1], W);
            if (spin)
                for (int k = 0; k < 3; ++k)
                    cudaMemcpyAsync(segJ[3 * m + k], Jw[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
        for (int m = len - 1; m >= 0 && st == GRPIC_OK; --m) {
            // seed: lamF (adjoint of F^{n+1}) += wL dflux/dF^{n+1}
            for (int k = 0; k < 6; ++k) cudaMemsetAsync(aux[k], 0, fn * sizeof(double), s);
            cudaMemcpyAsync(dSegF, seg[m + 1].F, sizeof(double *) * 6, cudaMemcpyHostToDevice, s);
            flux_seed<<<(ctx->g.nth + 127) / 128, 128, 0, s>>>(A, dSegF, i_horizon, dth, wL, dAux);
            aux_T<<<gfull, blk, 0, s>>>(A, dAux, dLamF);
            // fields: lamF -> lamF2 (adjoint of F^n through the field update), lamJ
            if (spin) {
                // the update of step m again, every stage kept
                if (launch_field64_stages(ctx, seg[m].F, &segJ[3 * m], Ystage.data(), ld, s) != cudaSuccess) {
                    st = GRPIC_ECUDA;
                    break;
                }
                cudaMemcpyAsync(spf.Xn, seg[m].F, sizeof(double *) * 6, cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(spf.J, &segJ[3 * m], sizeof(double *) * 3, cudaMemcpyHostToDevice, s);
            }
            st = field_adjoint(ctx, lamF, lamF2, lamJ, work.data(), ld, s, dptrs, spin ? &spf : nullptr);
            if (st != GRPIC_OK) break;
            // particles
            PAdjArgs P;
            P.g = ctx->g;
            P.dt = ctx->prm.dt;
            P.n_iter = ctx->prm.n_push_iter;
            P.ift = trapezoid_ift ? 1 : 0;
            for (int k = 0; k < 4; ++k) {
                P.qm[k] = ctx->prm.q_over_m[k];
                P.qw[k] = ctx->prm.q_weight[k];
                P.massive[k] = ctx->prm.massive[k];
            }
            P.n = np;
            for (int k = 0; k < 5; ++k) {
                P.x[k] = seg[m].x[k];
                P.lam1[k] = lamP[k];
                P.lam0[k] = lamP2[k];
            }
            P.tape = tape + (size_t)m * TW * (size_t)np;
            P.tape_ld = np;
            P.tag0 = seg[m].tag;
            P.tag1 = seg[m + 1].tag;
            for (int k = 0; k < 6; ++k) {
                P.F[k] = seg[m].F[k];
                P.lamF[k] = lamF2[k];
            }
            for (int k = 0; k < 3; ++k) P.lamJ[k] = lamJ[k];
            P.ld = ld;
            P.La = spin ? Lap : nullptr;
            if (np > 0 && spin) particle_adjoint<true><<<(unsigned)((np + 127) / 128), 128, 0, s>>>(P);
            if (np > 0 && !spin) particle_adjoint<false><<<(unsigned)((np + 127) / 128), 128, 0, s>>>(P);
            if (spin && np > 0) {
                unsigned nb = (unsigned)std::min<int64_t>((np + 255) / 256, 4 * 152);
                sum_into<<<nb, 256, 0, s>>>(Lap, np, Ladev);
            }
            if (cudaGetLastError() != cudaSuccess) st = GRPIC_ECUDA;
            for (int k = 0; k < 5; ++k) std::swap(lamP[k], lamP2[k]);
            // lamF <- lamF2
            for (int k = 0; k < 6; ++k) cudaMemcpyAsync(lamF[k], lamF2[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
    }
    for (int k = 0; k < 5; ++k) cudaMemcpyAsync(grad_p[k], lamP[k], np * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (grad_f)
        for (int k = 0; k < 6; ++k)
            if (grad_f[k]) cudaMemcpyAsync(grad_f[k], lamF[k], fn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (spin) cudaMemcpyAsync(dL_da, Ladev, sizeof(double), cudaMemcpyDeviceToHost, s);
    // a particle the forward refused (range, non-finite) is reported like the step does
    int hst = 0;
    cudaMemcpyAsync(&hst, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    ctx->keys_valid = 0;
    ctx->hist_valid = 0;
    cleanup();
    if (cudaGetLastError() != cudaSuccess && st == GRPIC_OK) st = GRPIC_ECUDA;
    if (st == GRPIC_OK && hst != 0) st = (grpic_status)hst;
    return st;
}
