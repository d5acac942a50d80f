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

// X^i, U_i of Eq. particle-eom from (r, sin theta, cos theta) without the
// metric's derivatives as separate fields: gamma^{jk} = rho^-2 [(a^2 + r^2,
// a, 1, 1/sin^2) in (rr, r phi, th th, phi phi)] - beta dr dr, so with
// P = (a^2 + r^2) u_r^2 + 2 a u_r u_ph + u_th^2 + u_ph^2 / sin^2 the forms in u
// collect into gamma^{jk} u_j u_k = P / rho^2 - beta u_r^2,
// d_r gamma^{jk} u_j u_k = u_r^2 (z - d_r beta) - 2 r P / rho^4 and
// d_th gamma^{jk} u_j u_k = -d_th rho^2 P / rho^4 - d_th beta u_r^2
//                           - 2 sin cos u_ph^2 / (rho^2 sin^4)
template <typename T>
__device__ __forceinline__ void geo_rhs_direct(T a, T eps, T r, T s, T c, T ur, T ut, T up, RhsT<T> &f)
{
    const T a2 = a * a, r2 = r * r;
    const T ir = rcp_t(r2 + a2 * c * c);
    const T ir2 = ir * ir;
    const T z = T(2) * r * ir;
    const T iopz = rcp_t(T(1) + z);
    const T alpha = sqrt_t(iopz);
    const T beta = z * iopz;
    const T is2 = rcp_t(s * s);
    const T drho_t = T(-2) * a2 * c * s;
    const T dz_r = T(2) * ir * (T(1) - T(2) * r2 * ir);
    const T dz_t = T(-2) * r * drho_t * ir2;
    const T ka = T(-0.5) * alpha * iopz, kb = iopz * iopz;
    const T db_r = kb * dz_r, db_t = kb * dz_t;
    const T ur2 = ur * ur, up2 = up * up;
    const T P = (a2 + r2) * ur2 + T(2) * a * ur * up + ut * ut + up2 * is2;
    const T au0 = sqrt_t(eps + ir * P - beta * ur2);  // alpha u^0
    const T iu0 = alpha * rcp_t(au0);
    const T grp = a * ir;
    f.xr = (((a2 + r2) * ir - beta) * ur + grp * up) * iu0 - beta;
    f.xt = ir * ut * iu0;
    f.xp = (grp * ur + ir * is2 * up) * iu0;
    const T h = T(0.5) * iu0;
    f.ur = -au0 * ka * dz_r + ur * db_r - h * (ur2 * (z - db_r) - T(2) * r * ir2 * P);
    f.ut = -au0 * ka * dz_t + ur * db_t - h * (-drho_t * ir2 * P - db_t * ur2 - T(2) * s * c * ir * is2 * is2 * up2);
}

// The same right-hand side in FP32 with a^2 given and the products ordered
// for fused multiply-adds; 1/(1+z) lies in (0, 1], so alpha takes the
// hardware reciprocal square root without a range test.
__device__ __forceinline__ void geo_rhs_direct32(float a, float a2, float eps, float r, float s, float c, float ur,
                                                 float ut, float up, RhsT<float> &f)
{
    const float r2 = r * r;
    const float ir = __fdividef(1.0f, fmaf(a2 * c, c, r2));
    const float ir2 = ir * ir;
    const float z = (r + r) * ir;
    const float iopz = __fdividef(1.0f, 1.0f + z);
    const float alpha = iopz * rsqrtf(iopz);
    const float beta = z * iopz;
    const float is2 = __fdividef(1.0f, s * s);
    const float drho_t = -2.0f * a2 * (c * s);
    const float dz_r = (ir + ir) * fmaf(-2.0f * r2, ir, 1.0f);
    const float dz_t = -2.0f * r * drho_t * ir2;
    const float kb = iopz * iopz;
    const float db_r = kb * dz_r, db_t = kb * dz_t;
    const float ur2 = ur * ur, up2 = up * up;
    const float ar2 = a2 + r2;
    const float P = fmaf(ar2, ur2, fmaf((a + a) * ur, up, fmaf(ut, ut, up2 * is2)));
    const float au0 = sqrt_t(fmaf(ir, P, fmaf(-beta, ur2, eps)));  // alpha u^0
    const float iu0 = alpha * __fdividef(1.0f, au0);
    const float grp = a * ir;
    f.xr = fmaf(fmaf(fmaf(ar2, ir, -beta), ur, grp * up), iu0, -beta);
    f.xt = ir * ut * iu0;
    f.xp = fmaf(grp, ur, ir * is2 * up) * iu0;
    const float h = 0.5f * iu0;
    // -alpha u^0 d alpha = alpha u^0 (alpha / (2 (1+z))) dz
    const float kad = 0.5f * alpha * iopz * au0;
    f.ur = fmaf(kad, dz_r, fmaf(ur, db_r, -h * fmaf(ur2, z - db_r, -2.0f * r * ir2 * P)));
    f.ut = fmaf(kad, dz_t, fmaf(ur, db_t, h * fmaf(drho_t * ir2, P, fmaf(db_t, ur2, 2.0f * s * c * ir * is2 * is2 * up2))));
}

}  // namespace grpic
