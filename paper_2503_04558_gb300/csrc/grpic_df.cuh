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

// 1/x: y0 ~ 1/x.hi (2 ulp), y = y0 + y0 e with the residual e = 1 - x y0
// (|e| ~ 2^-22) formed as fma(-x.hi, y0, 1) - x.lo y0: the fused
// multiply-add's single rounding of a value that small is below 2^-46, so
// y carries about 2^-44 relative error (the square of e and the rounding of
// y0 e), far under the FP32 rounding its consumers take
__device__ __forceinline__ df rcp_t(const df &x)
{
    const float y0 = __fdividef(1.0f, x.hi);
    const float e = fmaf(-x.lo, y0, fmaf(-x.hi, y0, 1.0f));
    return fast_two_sum(y0, __fmul_rn(e, y0));
}

__device__ __forceinline__ df operator/(const df &a, const df &b) { return a * rcp_t(b); }

// sqrt(x) for x >= 0 (0 otherwise): s0 = x.hi rsqrt(x.hi), s = s0 + (x - s0^2) / (2 s0)
// with the residual x - s0^2 = fma(-s0, s0, x.hi) + x.lo (exact to 2^-46 of x)
__device__ __forceinline__ df sqrt_t(const df &x)
{
    if (!(x.hi > 0.0f)) return df(0.0f);
    const float y0 = rsqrtf(x.hi);
    const float s0 = __fmul_rn(x.hi, y0);
    const float e = __fadd_rn(fmaf(-s0, s0, x.hi), x.lo);
    return fast_two_sum(s0, __fmul_rn(e, __fmul_rn(0.5f, y0)));
}

// 2^k x: exact scaling of both parts
__device__ __forceinline__ df scale2(const df &x, float p2) { return df(__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)); }

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

// a + b for a pair and a float
__device__ __forceinline__ df add_f(const df &a, float b)
{
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// sin, cos of (theta0 + d) from those of theta0 for a step |d| <= 0.1 (one
// theta cell or less): with e_c = 1 - cos d and e_s = 1 - sin(d)/d,
//   sin = s0 + c0 d - (s0 e_c + c0 d e_s),  cos = c0 - s0 d - (c0 e_c - s0 d e_s);
// the leading terms in pair arithmetic, the corrections (d^2 / 2 of the
// leading terms' size) in FP32 from their Taylor series to d^8 (truncation
// below d^10 / 10! = 3e-17), so their rounding stays below 2^-24 d^2 / 2 of
// the leading terms: 2^-44 at d = 1.5e-3 (2048 theta cells), 2^-31 at d = 0.1
__device__ __forceinline__ void sincos_shift_df(const df &s0, const df &c0, const df &d, df &s, df &c)
{
    const float x = d.hi, x2 = x * x;
    const float ec = x2 * fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 40320.0f, 1.0f / 720.0f), -1.0f / 24.0f), 0.5f);
    const float es = x2 * fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 362880.0f, 1.0f / 5040.0f), -1.0f / 120.0f),
                               1.0f / 6.0f);
    const float xes = x * es;
    s = add_f(s0 + c0 * d, -fmaf(s0.hi, ec, c0.hi * xes));
    c = add_f(c0 - s0 * d, -fmaf(c0.hi, ec, -s0.hi * xes));
}

}  // namespace grpic
