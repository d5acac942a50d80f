// grpic_shape3.cuh -- the third-order particle shape of Sec. 2.3 (a
// configuration option there): the cubic B-spline in logical units,
//   W3(x) = 2/3 - x^2 + |x|^3/2 (|x| < 1),  (2 - |x|)^3 / 6 (1 <= |x| < 2),
// S = W3(x1 - i) W3(x2 - j) on each staggered lattice, for the field
// interpolation (4 x 4 taps) and the Esirkepov deposit (Eq. esirkepov-decomp
// over the 5 x 5 vertices around both positions, Eq. j-phi-deposit).
//
// Rows past the polar axis are the mirror rows of the relabelling (r, -theta,
// phi + pi) of the same point: the theta components (D^theta, B^theta,
// J^theta) change sign there, the others do not; the axis rows are their own
// mirrors.  Interpolation reads the mirror rows with that parity, the
// deposit adds into them with it (which keeps the continuity of the
// half-width axis cells exact).  Columns: the two guard columns on each side
// hold what the interpolation needs; deposits past them (a particle leaving
// through r_out) are dropped.
#pragma once

#include "grpic_internal.cuh"

namespace grpic {

__device__ __forceinline__ double w3(double d)
{
    d = fabs(d);
    if (d < 1.0) return 2.0 / 3.0 - d * d + 0.5 * d * d * d;
    if (d < 2.0) {
        const double e = 2.0 - d;
        return e * e * e * (1.0 / 6.0);
    }
    return 0.0;
}

// the four weights W3(t + 1), W3(t), W3(t - 1), W3(t - 2) of the taps at
// floor(x) - 1 .. floor(x) + 2 for t = x - floor(x) in [0, 1), without branches:
// (1-t)^3/6, 2/3 - t^2 + t^3/2, 2/3 - (1-t)^2 + (1-t)^3/2, t^3/6
__device__ __forceinline__ void w3_taps(double t, double w[4])
{
    const double u = 1.0 - t, t2 = t * t, u2 = u * u;
    w[0] = u2 * u * (1.0 / 6.0);
    w[1] = 2.0 / 3.0 - t2 + 0.5 * t2 * t;
    w[2] = 2.0 / 3.0 - u2 + 0.5 * u2 * u;
    w[3] = t2 * t * (1.0 / 6.0);
}

// one lattice's taps at a point: the first tap index floor(x) - 1 and the weights
struct Taps3 {
    int i;
    double w[4];
};
__device__ __forceinline__ void taps3(double x, Taps3 &T)
{
    const double f = floor(x);
    T.i = (int)f - 1;
    w3_taps(x - f, T.w);
}

// W3(x - (b + k)) for k = 0..4: the taps placed in a window starting at b
// (taps that fall outside the window carry W3 = 0 there, as their distance
// is 2 or more)
__device__ __forceinline__ void w3_window5(double x, int b, double S[5])
{
    Taps3 T;
    taps3(x, T);
    const int o = T.i - b;  // window position of the first tap
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int a = k - o;
        S[k] = a == 0 ? T.w[0] : (a == 1 ? T.w[1] : (a == 2 ? T.w[2] : (a == 3 ? T.w[3] : 0.0)));
    }
}

// mirror of row j (integer rows theta_j, or half rows theta_{j+1/2})
__device__ __forceinline__ int mirror_row(int j, bool half_t, int nth, bool &flip)
{
    const int top = half_t ? nth - 1 : nth;
    flip = false;
    if (j < 0) {
        flip = true;
        return half_t ? -1 - j : -j;
    }
    if (j > top) {
        flip = true;
        return half_t ? 2 * nth - 1 - j : 2 * nth - j;
    }
    return j;
}

// a component from its lattice's taps in r (R) and theta (T)
__device__ __forceinline__ double gather3t(const double *__restrict__ F, int64_t ld, int nth, const Taps3 &R,
                                           const Taps3 &T, bool half_t, double par)
{
    double v = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        bool flip;
        const int jj = mirror_row(T.i + b, half_t, nth, flip);
        const double *row = F + (size_t)jj * ld + (R.i + NG);
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) s += R.w[a] * __ldg(row + a);
        v += T.w[b] * (flip ? par : 1.0) * s;
    }
    return v;
}

// the six fields at the particle (D^r, D^th, D^ph, B^r, B^th, B^ph); the
// components share two r lattices (integer, half) and two theta lattices, so
// four tap sets serve all six
__device__ __forceinline__ void gather3_fields(const double *D0, const double *D1, const double *D2, const double *B0,
                                               const double *B1, const double *B2, int64_t ld, int nth, double x1,
                                               double x2, double Dv[3], double Bv[3])
{
    Taps3 r0, rh, t0, th;
    taps3(x1, r0);
    taps3(x1 - 0.5, rh);
    taps3(x2, t0);
    taps3(x2 - 0.5, th);
    Dv[0] = gather3t(D0, ld, nth, rh, t0, false, 1.0);
    Dv[1] = gather3t(D1, ld, nth, r0, th, true, -1.0);
    Dv[2] = gather3t(D2, ld, nth, r0, t0, false, 1.0);
    Bv[0] = gather3t(B0, ld, nth, r0, th, true, 1.0);
    Bv[1] = gather3t(B1, ld, nth, rh, t0, false, -1.0);
    Bv[2] = gather3t(B2, ld, nth, rh, th, true, 1.0);
}

__device__ __forceinline__ void fold_add3(double *F, int64_t ld, int nr, int nth, int i, int j, bool half_t, double odd,
                                          double v)
{
    if (v == 0.0 || i < -NG || i > nr + NG - 1) return;
    bool flip;
    const int jj = mirror_row(j, half_t, nth, flip);
    atomicAdd(F + (size_t)jj * ld + (i + NG), flip ? odd * v : v);
}

// integrated currents of one move from (x1a, x2a) to (x1b, x2b) (logical,
// at most one cell apart in each direction): J^r A (J0), J^theta A (J1),
// J^phi dV (J2)
__device__ __forceinline__ void deposit3(int nr, int nth, int64_t ld, double *J0, double *J1, double *J2, double qw,
                                         double dt, double x1a, double x2a, double x1b, double x2b, double dphi)
{
    const int fa = (int)floor(x1a), fb = (int)floor(x1b);
    const int b1 = (fa < fb ? fa : fb) - 1;
    const int ga = (int)floor(x2a), gb = (int)floor(x2b);
    const int b2 = (ga < gb ? ga : gb) - 1;
    double S0r[5], S1r[5], S0t[5], S1t[5];
    w3_window5(x1a, b1, S0r);
    w3_window5(x1b, b1, S1r);
    w3_window5(x2a, b2, S0t);
    w3_window5(x2b, b2, S1t);
    const double cr = -qw / (2.0 * dt), cp = qw * dphi / dt;
    // J^r A at faces b1 + k + 1/2 (k = 0..3): prefix sums of (S1r - S0r) (S1t + S0t)
    double Pr = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Pr += S1r[k] - S0r[k];
#pragma unroll
        for (int l = 0; l < 5; ++l) fold_add3(J0, ld, nr, nth, b1 + k, b2 + l, false, 1.0, cr * Pr * (S1t[l] + S0t[l]));
    }
    double Pt = 0.0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        Pt += S1t[l] - S0t[l];
#pragma unroll
        for (int k = 0; k < 5; ++k) fold_add3(J1, ld, nr, nth, b1 + k, b2 + l, true, -1.0, cr * (S1r[k] + S0r[k]) * Pt);
    }
    // J^phi dV weights S1r S1t / 3 + S1r S0t / 6 + S0r S1t / 6 + S0r S0t / 3,
    // factored per row: S1r A_t + S0r B_t
    double At[5], Bt[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        At[l] = cp * (S1t[l] * (1.0 / 3.0) + S0t[l] * (1.0 / 6.0));
        Bt[l] = cp * (S1t[l] * (1.0 / 6.0) + S0t[l] * (1.0 / 3.0));
    }
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int l = 0; l < 5; ++l) fold_add3(J2, ld, nr, nth, b1 + k, b2 + l, false, 1.0, S1r[k] * At[l] + S0r[k] * Bt[l]);
}

}  // namespace grpic
