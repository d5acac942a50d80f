// grpic_df.cuh -- double-FP32 ("double-float") arithmetic for the near-horizon
// metric island of the FP32 form.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  Built from the error-free transformations
// TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2), FastTwoSum (Dekker 1971) and
// TwoProd through the fused multiply-add; the reciprocal and the square root
// take one Newton step in pair arithmetic from the hardware FP32 estimate.
// Sums use the cheap form (relative error ~2^-46 of max(|a|, |b|)), which is
// what FP64 subtraction would deliver after rounding to the FP32 that the
// right-hand sides of the FP32 form consume.
//
// All float operations inside the transformations go through __fadd_rn /
// __fmul_rn / fmaf so that the compiler cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace grpic {

struct df {
    float hi, lo;
    __host__ __device__ df() {}
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ df(float x) : hi(x), lo(0.0f) {}
    __device__ __forceinline__ df(int x) : hi((float)x), lo(0.0f) {}  // small integers (exact)
    // literals of the metric formulas (0.5, 2, ...) are exact in float; a
    // general double splits into its leading float and the rounded remainder
    __device__ __forceinline__ df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float v = __fadd_rn(s, -a);
    float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -v)), __fadd_rn(b, -v));
    return df(s, e);
}

__device__ __forceinline__ df fast_two_sum(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    return df(s, __fadd_rn(b, -__fadd_rn(s, -a)));
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    return df(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df operator+(const df &a, const df &b)
{
    df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(const df &a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(const df &a, const df &b) { return a + (-b); }

__device__ __forceinline__ df operator*(const df &a, const df &b)
{
    df p = two_prod(a.hi, b.hi);
    float t = fmaf(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

__device__ __forceinline__ df mul(const df &a, float b)
{
    df p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// 1/x: y0 ~ 1/x.hi (2 ulp), y = y0 + y0 (1 - x y0) with the residual in pairs
__device__ __forceinline__ df rcp_t(const df &x)
{
    float y0 = __fdividef(1.0f, x.hi);
    df xy = mul(x, y0);
    df e = df(1.0f) - xy;
    return fast_two_sum(y0, __fmul_rn(e.hi, y0));
}

__device__ __forceinline__ df operator/(const df &a, const df &b) { return a * rcp_t(b); }

// sqrt(x) for x >= 0 (0 otherwise): s0 = x.hi rsqrt(x.hi), s = s0 + (x - s0^2) / (2 s0)
__device__ __forceinline__ df sqrt_t(const df &x)
{
    if (!(x.hi > 0.0f)) return df(0.0f);
    float y0 = rsqrtf(x.hi);
    float s0 = __fmul_rn(x.hi, y0);
    df e = x - two_prod(s0, s0);
    return fast_two_sum(s0, __fmul_rn(e.hi, __fmul_rn(0.5f, y0)));
}

// sin/cos of a pair through FP64 (the island takes this only for angle steps
// beyond the Taylor range of sincos_shift_df, which the push does not reach
// on grids with n_theta >= 32)
__device__ __forceinline__ void sincos_t(const df &x, df *s, df *c)
{
    double sd, cd;
    sincos((double)x.hi + (double)x.lo, &sd, &cd);
    *s = df(sd);
    *c = df(cd);
}

__device__ __forceinline__ float fabs_hi(const df &x) { return fabsf(x.hi); }

// split of a double constant into a pair at compile time
constexpr df df_const(double x) { return df((float)x, (float)(x - (double)(float)x)); }

// sin, cos of (theta0 + d) from those of theta0, |d| small: the Taylor series
// of sin d and cos d to d^9 and d^8 (truncation below 1e-15 for |d| <= 0.1)
__device__ __forceinline__ void sincos_shift_df(const df &s0, const df &c0, const df &d, df &s, df &c)
{
    constexpr df i6 = df_const(1.0 / 6.0), i20 = df_const(1.0 / 20.0), i42 = df_const(1.0 / 42.0),
                 i72 = df_const(1.0 / 72.0), i12 = df_const(1.0 / 12.0), i30 = df_const(1.0 / 30.0),
                 i56 = df_const(1.0 / 56.0);
    df d2 = d * d;
    df one(1.0f);
    df sd = d * (one - d2 * i6 * (one - d2 * i20 * (one - d2 * i42 * (one - d2 * i72))));
    df cd = one - mul(d2, 0.5f) * (one - d2 * i12 * (one - d2 * i30 * (one - d2 * i56)));
    s = s0 * cd + c0 * sd;
    c = c0 * cd - s0 * sd;
}

}  // namespace grpic
