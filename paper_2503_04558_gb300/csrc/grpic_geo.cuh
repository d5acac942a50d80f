// grpic_geo.cuh -- Kerr-Schild metric pieces needed by the pusher, templated
// on the arithmetic type (double for the FP64 path and the FP64 islands of the
// FP32 form, float for the FP32 form).
//
// KSGeo holds alpha, beta^r, gamma^{ij} and their analytic r and theta
// derivatives (App. A, Eqs. gamma-inverse, ks-alpha-beta); geo_rhs assembles
// the right-hand sides X^i, U_i of Eq. particle-eom (without the Lorentz force).
#pragma once

#include "grpic_internal.cuh"

namespace grpic {

template <typename T>
struct KSGeo {
    T alpha, beta, grr, grp, gtt, gpp;
    T da_r, da_t, db_r, db_t;
    T dgrr_r, dgrr_t, dgrp_r, dgrp_t, dgtt_r, dgtt_t, dgpp_r, dgpp_t;
    T rho2, ir, opz;  // rho^2, 1/rho^2, 1 + z (for the lower metric of the Boris step)
};

template <typename T>
struct RhsT {
    T xr, xt, xp, ur, ut;
};

// FP32 (the FP32 form, whose error budget is 1e-4 against FP64): hardware
// approximations with a relative error of a few ulp for reciprocal and square
// root; sin/cos keep the accurate sincosf because near the polar axis
// sin(theta) needs relative accuracy (the fast __sincosf has an absolute error
// of ~2^-21).  FP64 (the FP64 island of the FP32 form): reciprocal and square
// root from an FP32 seed refined by two Newton steps in FP64 (relative error
// below 2^-52 for the normal range used here), sin/cos from the library.
__device__ __forceinline__ void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ double rcp_t(double x)
{
    double y = (double)__frcp_rn((float)x);
    y = y * (2.0 - x * y);
    return y * (2.0 - x * y);
}
__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double sqrt_t(double x)
{
    if (!(x > 0.0)) return 0.0;
    double y = (double)rsqrtf((float)x);       // 1/sqrt(x), 2^-22
    y = y * (1.5 - 0.5 * x * y * y);           // 2^-44
    y = y * (1.5 - 0.5 * x * y * y);           // full precision
    double s = x * y;
    return s + 0.5 * y * (x - s * s);          // one correction of the root itself
}
__device__ __forceinline__ float sqrt_t(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// sin, cos of (theta0 + d) from sin, cos of theta0 and a short Taylor series
// of sin d, cos d; for |d| <= 0.05 the truncated terms are below 1e-17 in
// FP64 and below 3e-12 (to d^5 and d^4) in FP32.
template <typename T>
__device__ __forceinline__ void sincos_shift(T s0, T c0, T d, T &s, T &c)
{
    T d2 = d * d;
    T sd = d * (T(1) - d2 * (T(1) / T(6)) * (T(1) - d2 * (T(1) / T(20)) * (T(1) - d2 * (T(1) / T(42)))));
    T cd = T(1) - d2 * T(0.5) * (T(1) - d2 * (T(1) / T(12)) * (T(1) - d2 * (T(1) / T(30)) * (T(1) - d2 * (T(1) / T(56)))));
    s = s0 * cd + c0 * sd;
    c = c0 * cd - s0 * sd;
}
template <>
__device__ __forceinline__ void sincos_shift<float>(float s0, float c0, float d, float &s, float &c)
{
    const float d2 = d * d;
    const float sd = d * fmaf(d2, fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    const float cd = fmaf(d2, fmaf(d2, 1.0f / 24.0f, -0.5f), 1.0f);
    s = fmaf(s0, cd, c0 * sd);
    c = fmaf(c0, cd, -s0 * sd);
}

// metric + derivatives at (r, theta) given sin/cos of theta
template <typename T>
__device__ __forceinline__ void ks_geo_sc(T a, T r, T s, T c, KSGeo<T> &m)
{
    T a2 = a * a, r2 = r * r;
    T rho2 = r2 + a2 * c * c;
    T ir = rcp_t(rho2);
    T ir2 = ir * ir;
    T z = T(2) * r * ir;
    T iopz = rcp_t(T(1) + z);
    m.rho2 = rho2;
    m.ir = ir;
    m.opz = T(1) + z;
    m.alpha = sqrt_t(iopz);
    m.beta = z * iopz;
    T is2 = rcp_t(s * s);
    m.grr = (a2 + r2) * ir - m.beta;
    m.grp = a * ir;
    m.gtt = ir;
    m.gpp = ir * is2;
    T drho_t = T(-2) * a2 * c * s;
    T dz_r = T(2) * ir * (T(1) - T(2) * r2 * ir);
    T dz_t = T(-2) * r * drho_t * ir2;
    T ka = T(-0.5) * m.alpha * iopz;  // d alpha / dz
    T kb = iopz * iopz;               // d beta / dz
    m.da_r = ka * dz_r;
    m.da_t = ka * dz_t;
    m.db_r = kb * dz_r;
    m.db_t = kb * dz_t;
    m.dgrr_r = T(2) * r * ir - (a2 + r2) * T(2) * r * ir2 - m.db_r;
    m.dgrr_t = -(a2 + r2) * drho_t * ir2 - m.db_t;
    m.dgrp_r = -a * T(2) * r * ir2;
    m.dgrp_t = -a * drho_t * ir2;
    m.dgtt_r = T(-2) * r * ir2;
    m.dgtt_t = -drho_t * ir2;
    m.dgpp_r = T(-2) * r * ir2 * is2;
    m.dgpp_t = -drho_t * ir2 * is2 - T(2) * s * c * ir * is2 * is2;
}

template <typename T>
__device__ __forceinline__ void ks_geo(T a, T r, T th, KSGeo<T> &m)
{
    T s, c;
    sincos_t(th, &s, &c);
    ks_geo_sc(a, r, s, c, m);
}

// X^i = gamma^{ij} u_j / u^0 - beta^i,
// U_i = -alpha u^0 d_i alpha + u_k d_i beta^k - u_j u_k d_i gamma^{jk} / (2 u^0)
template <typename M, typename T>
__device__ __forceinline__ void geo_rhs_m(const KSGeo<M> &m, T eps, T ur, T ut, T up, RhsT<T> &f)
{
    T grr = (T)m.grr, grp = (T)m.grp, gtt = (T)m.gtt, gpp = (T)m.gpp, alpha = (T)m.alpha;
    T uu = grr * ur * ur + T(2) * grp * ur * up + gtt * ut * ut + gpp * up * up;
    T au0 = sqrt_t(eps + uu);  // alpha u^0
    T iu0 = alpha * rcp_t(au0);  // 1 / u^0
    f.xr = (grr * ur + grp * up) * iu0 - (T)m.beta;
    f.xt = gtt * ut * iu0;
    f.xp = (grp * ur + gpp * up) * iu0;
    T h = T(0.5) * iu0;
    f.ur = -au0 * (T)m.da_r + ur * (T)m.db_r -
           h * (ur * ur * (T)m.dgrr_r + T(2) * ur * up * (T)m.dgrp_r + ut * ut * (T)m.dgtt_r + up * up * (T)m.dgpp_r);
    f.ut = -au0 * (T)m.da_t + ur * (T)m.db_t -
           h * (ur * ur * (T)m.dgrr_t + T(2) * ur * up * (T)m.dgrp_t + ut * ut * (T)m.dgtt_t + up * up * (T)m.dgpp_t);
}

// The right-hand side of the FP32 form and of the FP64 path, split into the
// quantities of the point (r, sin theta, cos theta) -- shared by the Boris
// step and the right-hand side at x^n -- and the part that depends on u.  With
//   P = (a^2 + r^2) u_r^2 + 2 a u_r u_ph + u_th^2 + u_ph^2 / sin^2,
// gamma^{jk} u_j u_k = P / rho^2 - beta u_r^2 (gamma^{jk} of App. A), so that
// with Q = eps + gamma^{jk} u_j u_k: alpha u^0 = sqrt(Q), 1/u^0 = alpha / sqrt(Q).
// The force terms of Eq. particle-eom collect, with h = 1 / (2 u^0),
// d_r z = 2/rho^2 - z^2 and d_th z = -z E (E = d_th rho^2 / rho^2), as
//   -alpha u^0 d_i alpha + u_r d_i beta^r + h u_r^2 d_i beta^r = K d_i z,
//   K = (1+z)^-1 (h Q + (1+z)^-1 u_r (1 + h u_r))
// (alpha^2 = (1+z)^-1, d_i alpha = -alpha^3 d_i z / 2, d_i beta^r =
// (1+z)^-2 d_i z), and the remaining derivatives of P / rho^2 give
//   U_r  = K d_r z + h z (P / rho^2 - u_r^2),
//   U_th = E (h P / rho^2 - K z) + (1/u^0) rho^-2 sin cos sin^-4 u_ph^2
// (d_th sin^-2 = -2 sin cos / sin^4).  1/(1+z) lies in (0, 1].
//
// Per type: the reciprocal and reciprocal square root the right-hand side
// takes (FP32: the hardware approximations; FP64: an FP32 seed refined by
// two Newton steps, the residual formed by a fused multiply-add, relative
// error a few ulp of FP64; arguments within FP32's normal range) and the
// fused multiply-add
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_fast(double x) { return rcp_t(x); }
__device__ __forceinline__ float rsqrt_fast(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_fast(double x)
{
    double y = (double)rsqrtf((float)x);  // 2^-22
    double e = fma(-x * y, y, 1.0);       // 1 - x y^2
    y = fma(0.5 * y, e, y);               // 2^-43
    e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
struct PtT {
    T s, rho2, ir, z, opz, al, iopz, beta, s2, is2, ar2, cs, E;
};
using Pt32 = PtT<float>;

template <typename T>
__device__ __forceinline__ PtT<T> pointT(T a2, T m2a2, T r, T s, T c)
{
    PtT<T> m;
    const T r2 = r * r;
    m.s = s;
    m.rho2 = fmat(a2 * c, c, r2);
    m.ir = rcp_fast(m.rho2);
    m.z = (r + r) * m.ir;
    m.opz = T(1) + m.z;
    m.al = rsqrt_fast(m.opz);
    m.iopz = m.al * m.al;
    m.beta = m.z * m.iopz;
    m.s2 = s * s;
    m.is2 = rcp_fast(m.s2);
    m.ar2 = a2 + r2;
    m.cs = c * s;
    m.E = m2a2 * m.cs * m.ir;  // m2a2 = -2 a^2
    return m;
}

__device__ __forceinline__ Pt32 point32(float a2, float m2a2, float r, float s, float c)
{
    return pointT<float>(a2, m2a2, r, s, c);
}

// aup = a u_ph (u_ph is fixed during the correctors)
template <typename T>
__device__ __forceinline__ void rhsT(const PtT<T> &m, T a, T eps, T ur, T ut, T up, T aup, RhsT<T> &f)
{
    const T ur2 = ur * ur;
    const T is2up = m.is2 * up;
    const T is2up2 = is2up * up;
    const T w = fmat(m.ar2, ur, aup);                          // (a^2 + r^2) u_r + a u_ph
    const T P = fmat(ur, w + aup, fmat(ut, ut, is2up2));
    const T irP = m.ir * P;
    const T Q = fmat(m.ir, P, fmat(-m.beta, ur2, eps));
    const T qq = rsqrt_fast(Q);
    const T iu0 = m.al * qq;                                   // 1 / u^0
    const T h = T(0.5) * iu0;
    const T iri = m.ir * iu0;
    f.xr = fmat(iu0, fmat(m.ir, w, -m.beta * ur), -m.beta);
    f.xt = iri * ut;
    f.xp = iri * fmat(a, ur, is2up);
    const T K = m.iopz * fmat(m.iopz * ur, fmat(h, ur, T(1)), h * Q);
    f.ur = fmat(K, fmat(-m.z, m.z, m.ir + m.ir), h * m.z * (irP - ur2));
    f.ut = fmat(m.E, fmat(-K, m.z, h * irP), iri * (m.cs * m.is2) * is2up2);
}

__device__ __forceinline__ void rhs32(const Pt32 &m, float a, float eps, float ur, float ut, float up, float aup,
                                      RhsT<float> &f)
{
    rhsT<float>(m, a, eps, ur, ut, up, aup, f);
}

// The same right-hand side from the upper metric's values given apart
// (the near-horizon island forms them in extended precision): with
// gamma^{rj} u_j, gamma^{phi j} u_j and G = gamma^{jk} u_j u_k, Q = eps + G,
// P / rho^2 = G + beta u_r^2, and the force terms as in rhs32.
struct GUp32 {
    float rr, rp, tt, pp;
};

__device__ __forceinline__ void rhs32g(const Pt32 &m, const GUp32 &g, float eps, float ur, float ut, float up,
                                       RhsT<float> &f)
{
    const float ur2 = ur * ur;
    const float gur = fmaf(g.rr, ur, g.rp * up);  // gamma^{rj} u_j
    const float gup = fmaf(g.rp, ur, g.pp * up);  // gamma^{phi j} u_j
    const float gtu = g.tt * ut;
    const float G = fmaf(gur, ur, fmaf(gtu, ut, gup * up));
    const float Q = G + eps;
    const float qq = rsqrtf(Q);
    const float iu0 = m.al * qq;
    const float h = 0.5f * iu0;
    const float iri = m.ir * iu0;
    f.xr = fmaf(iu0, gur, -m.beta);
    f.xt = iu0 * gtu;
    f.xp = iu0 * gup;
    const float irP = fmaf(m.beta, ur2, G);
    const float K = m.iopz * fmaf(m.iopz * ur, fmaf(h, ur, 1.0f), h * Q);
    f.ur = fmaf(K, fmaf(-m.z, m.z, m.ir + m.ir), h * m.z * (irP - ur2));
    f.ut = fmaf(m.E, fmaf(-K, m.z, h * irP), iri * (m.cs * m.is2) * (m.is2 * up * up));
}

}  // namespace grpic
