// grpic_push32.cu -- FP32 form of the push fused with the deposit.
//
// Same algorithm as the FP64 path (arXiv:2503.04558 Sec. 2.2-2.3): Boris at
// fields n, geodesic predictor + trapezoidal correctors, axis reflection,
// Esirkepov deposit.  What changes is the number format:
//   * a particle is an int32 cell key plus FP32 offsets (o1, o2) in [0, 1]
//     inside the cell (logical units) and FP32 covariant momenta -- in the
//     last theta row o2 holds q = (pi - theta) / dtheta, the distance to the
//     pole, so that theta near pi keeps FP32's relative precision as theta
//     near 0 does in row 0; the geodesic
//     is integrated for r - r_i (r_i the cell's inner edge) and for o2
//     (dx2/dt = X^th / dtheta), so the trapezoidal rule acts on r and theta as
//     in the paper while the position keeps FP32 precision relative to its
//     cell whatever the grid size;
//   * fields, tables and deposited currents are FP32;
//   * extended precision is kept for (i) the metric of particles in cells
//     whose inner edge lies below fp64_radius (the island near the horizon):
//     by default alpha, beta, gamma^ij and the lower metric in double-FP32
//     pairs, rounded to FP32 for the right-hand sides, with the metric's r and
//     theta derivatives (force terms only) in FP32; on request (island_arith)
//     the whole metric with its derivatives in native FP64; (ii) the corrector's
//     convergence test: after each corrector the change of the iterate is
//     measured (exactly, see below) and the iteration stops once it is below
//     the tolerance (at most n_push_iter correctors).
#include "grpic_geo.cuh"
#include "grpic_df.cuh"
#include "grpic_window.cuh"
#include "grpic_vay.cuh"

#include <algorithm>
#include <cmath>

namespace grpic {
namespace {

struct Push32Args {
    GridDev g;
    float dt;
    float idt, m_i2dt;  // 1 / dt, -1 / (2 dt)
    int n_iter;
    float tolf, tol_o2;  // push_tol; push_tol / dtheta (the theta test in offset units)
    float qm[4], qw[4];
    int massive[4];
    // per species (bit sp): massive (eps = 1 in u^0); massive and charged (the Boris step runs)
    unsigned massive_mask, boris_mask;
    double r64;
    int i64;  // first column whose inner edge is at or beyond fp64_radius
    int island_fp64;   // 1: native FP64 island, 0: double-FP32 pairs
    int use_tol;       // convergence test of the correctors
    float af, a2f, m2a2f, dthf, idthf, dx1f, idx1f;  // a, a^2, -2 a^2, dtheta, 1/dtheta, dx1, 1/dx1 in FP32
    df a_df, a2_df, dth_df;       // a, a^2, dtheta as float pairs
    const float *rcol2;  // r_i as (hi, lo) float pairs, index i + NG
    const float *rowsc;  // sin, cos theta_j as float pairs, index j
    int64_t n;
    const int64_t *d_count;
    int32_t *cell;
    float *o1, *o2, *u1, *u2, *u3;
    uint32_t *tag;
    // read through a permutation: slot p's particle comes from slot perm[p]
    // of the input arrays (the last sort's order, its data not yet moved);
    // live slots = *live, whose count goes to *count_out.  perm == nullptr:
    // the input arrays are the output arrays (in place).
    const int32_t *perm, *live;
    int64_t *count_out;
    // with perm: the particles of each old cell going in each direction
    // (direction-major, d * n_cells + cell; zeroed by the caller), the counts
    // of the next neighbour sort
    int32_t *cnt9;
    const int32_t *in_cell;
    const float *in_o1, *in_o2, *in_u1, *in_u2, *in_u3;
    const uint32_t *in_tag;
    // the field components D^r, D^th, D^ph, B^r, B^th, B^ph (c = 0..5) as
    // stencil quads (quad32_kernel), component c of the stencil at (is, js)
    // at element 6 ((js + 1) ld + is + NG) + c
    const float4 *Q;
    float *J0, *J1, *J2;
    int64_t ld;
    int ldi;  // ld as the 32-bit stride of the element offsets ((n_theta+1) ld < 2^31)
    const double *rcol;  // r at integer columns, index i + NG
    int32_t *keys;
    int32_t *count;
    int histogram;
    int *status;
    unsigned long long nr_recip;  // floor(2^64 / n_r) + 1
};

template <typename T>
struct KSPoint {
    T alpha, g_rr, g_rp, g_tt, g_pp, gi_rr, gi_rp, gi_tt, gi_pp, sqrtg;
};

template <typename T>
__device__ __forceinline__ void ks_point_t(T a, T r, T th, KSPoint<T> &m)
{
    T s, c;
    sincos_t(th, &s, &c);
    T s2 = s * s, a2 = a * a;
    T rho2 = r * r + a2 * c * c;
    T irho2 = T(1) / rho2;
    T z = T(2) * r * irho2;
    T opz = T(1) + z;
    T Dl = r * r + a2 - T(2) * r;
    T Sg = (r * r + a2) * (r * r + a2) - a2 * Dl * s2;
    m.alpha = sqrt_t(T(1) / opz);
    m.g_rr = opz;
    m.g_tt = rho2;
    m.g_pp = Sg * s2 * irho2;
    m.g_rp = -a * s2 * opz;
    m.gi_rr = (a2 + r * r) * irho2 - z / opz;
    m.gi_rp = a * irho2;
    m.gi_tt = irho2;
    m.gi_pp = irho2 / s2;
    m.sqrtg = rho2 * s * sqrt_t(opz);
}

// generalized Boris step in FP32 with a metric of type M
template <typename M>
__device__ __forceinline__ void boris32(const KSPoint<M> &mm, float qm, float dt, const float D[3], const float B[3],
                                        float u[3])
{
    float alpha = (float)mm.alpha, grr = (float)mm.g_rr, grp = (float)mm.g_rp, gtt = (float)mm.g_tt,
          gpp = (float)mm.g_pp;
    float irr = (float)mm.gi_rr, irp = (float)mm.gi_rp, itt = (float)mm.gi_tt, ipp = (float)mm.gi_pp;
    float sg = (float)mm.sqrtg;
    float Dl0 = grr * D[0] + grp * D[2], Dl1 = gtt * D[1], Dl2 = grp * D[0] + gpp * D[2];
    float h = (0.5f * qm * dt) * alpha;
    float um0 = u[0] + h * Dl0, um1 = u[1] + h * Dl1, um2 = u[2] + h * Dl2;
    float v0 = irr * um0 + irp * um2, v1 = itt * um1, v2 = irp * um0 + ipp * um2;
    // 1 / u0bar = alpha / sqrt(1 + u^- . v) (hardware reciprocal square root and
    // reciprocal: a few ulp, within the FP32 form's budget)
    float kt = h * rsqrtf(fmaf(um0, v0, fmaf(um1, v1, fmaf(um2, v2, 1.0f))));
    float t0 = kt * B[0], t1 = kt * B[1], t2 = kt * B[2];
    float tt = t0 * (grr * t0 + grp * t2) + t1 * (gtt * t1) + t2 * (grp * t0 + gpp * t2);
    float ks = __fdividef(2.0f, 1.0f + tt);
    float s0 = ks * t0, s1 = ks * t1, s2 = ks * t2;
    float w0 = um0 + sg * (v1 * t2 - v2 * t1);
    float w1 = um1 + sg * (v2 * t0 - v0 * t2);
    float w2 = um2 + sg * (v0 * t1 - v1 * t0);
    float x0 = irr * w0 + irp * w2, x1 = itt * w1, x2 = irp * w0 + ipp * w2;
    u[0] = um0 + sg * (x1 * s2 - x2 * s1) + h * Dl0;
    u[1] = um1 + sg * (x2 * s0 - x0 * s2) + h * Dl1;
    u[2] = um2 + sg * (x0 * s1 - x1 * s0) + h * Dl2;
}

// exp(x) - 1 for x = o1 dx1 in [0, dx1]: Taylor polynomial to x^6 when the
// cells are narrow (dx1 <= 0.1: truncation below x^7 / 7! = 2e-11, under
// FP32 rounding), the library function otherwise
__device__ __forceinline__ float expm1_cell(float x, float dx1)
{
    if (dx1 > 0.1f) return expm1f(x);
    return x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f + x * (1.0f / 120.0f + x * (1.0f / 720.0f))))));
}

// log(1 + y) for the relative move y of r against the cell's inner edge:
// alternating Taylor polynomial to y^8 for |y| <= 0.05 (truncation below
// y^9 / 9 = 2e-13), the library function otherwise
__device__ __forceinline__ float log1p_cell(float y)
{
    if (fabsf(y) > 0.05f) return log1pf(y);
    return y * (1.0f - y * (0.5f - y * (1.0f / 3.0f - y * (0.25f - y * (0.2f - y * (1.0f / 6.0f - y * (1.0f / 7.0f - y * 0.125f)))))));
}

// bilinear stencil from cell (i, j) and offsets; half_r / half_t stagger
// the component by half a cell in r / theta: the stencil's first column is
// and first row js (js = -1 below the first half row), f and gg its
// fractional offsets
struct Sq32 {
    int o;  // element offset of the stencil's quad
    float f, gg;
};

__device__ __forceinline__ void stencilq32(int ld, int i, int j, float o1, float o2, bool half_r, bool half_t, Sq32 &S)
{
    int is = i;
    float f = o1;
    if (half_r) {
        f = o1 - 0.5f;
        if (f < 0.0f) { f += 1.0f; is = i - 1; }
    }
    int js = j;
    float gg = o2;
    if (half_t) {
        gg = o2 - 0.5f;
        if (gg < 0.0f) { gg += 1.0f; js = j - 1; }
    }
    S.o = (js + 1) * ld + is + NG;
    S.f = f;
    S.gg = gg;
}

// the bilinear value of component c from its quad: along r on both rows,
// then along theta (the rows' axis parities are in the quad)
__device__ __forceinline__ float gatherq32(const float4 *__restrict__ Q, const Sq32 &S, int c)
{
    const float4 v = __ldg(Q + ((size_t)(unsigned)S.o * 6u + (unsigned)c));  // 32 x 32 -> 64-bit multiply
    const float x = fmaf(S.f, v.y - v.x, v.x), y = fmaf(S.f, v.w - v.z, v.z);
    return fmaf(S.gg, y - x, x);
}

// the six field components at the particle (Fig. Yee staggering): D^r and
// B^theta at (i+1/2, j), D^theta and B^r at (i, j+1/2), D^phi at (i, j),
// B^phi at (i+1/2, j+1/2); across the polar axis D^theta is odd, B^r and
// B^phi even (the quads hold the reflected rows)
__device__ __forceinline__ void gather_fields32(const Push32Args &A, int i, int j, float o1, float o2, float Dv[3],
                                                float Bv[3])
{
    Sq32 Sh0, S0h, S00, Shh;
    const int ld = A.ldi;
    stencilq32(ld, i, j, o1, o2, true, false, Sh0);
    stencilq32(ld, i, j, o1, o2, false, true, S0h);
    stencilq32(ld, i, j, o1, o2, false, false, S00);
    stencilq32(ld, i, j, o1, o2, true, true, Shh);
    Dv[0] = gatherq32(A.Q, Sh0, 0);
    Dv[1] = gatherq32(A.Q, S0h, 1);
    Dv[2] = gatherq32(A.Q, S00, 2);
    Bv[0] = gatherq32(A.Q, S0h, 3);
    Bv[1] = gatherq32(A.Q, Sh0, 4);
    Bv[2] = gatherq32(A.Q, Shh, 5);
}

// generalized Boris step in FP32 with the metric of type M at x^n (the lower
// metric is rebuilt from the quantities the geodesic evaluation keeps)
template <typename M>
__device__ __forceinline__ void boris_geo(const KSGeo<M> &m, M a, M r, M s, float qm, float dt, const float D[3],
                                          const float B[3], float u[3], int pusher)
{
    // gamma_rr = 1+z, gamma_thth = rho^2, gamma_phph = Sigma sin^2 / rho^2,
    // gamma_rph = -a sin^2 (1+z), sqrt(gamma) = rho^2 sin sqrt(1+z) = rho^2 sin / alpha
    M r2 = r * r;
    M s2 = s * s;
    M Dl = r2 + a * a - M(2) * r;
    M Sg = (r2 + a * a) * (r2 + a * a) - a * a * Dl * s2;
    KSPoint<float> mm;
    mm.alpha = (float)m.alpha;
    mm.g_rr = (float)m.opz;
    mm.g_tt = (float)m.rho2;
    mm.g_pp = (float)(Sg * s2 * m.ir);
    mm.g_rp = (float)(-a * s2 * m.opz);
    mm.gi_rr = (float)m.grr;
    mm.gi_rp = (float)m.grp;
    mm.gi_tt = (float)m.gtt;
    mm.gi_pp = (float)m.gpp;
    mm.sqrtg = (float)(m.rho2 * s * m.opz * m.alpha);  // rho^2 sin sqrt(1+z), sqrt(1+z) = (1+z) alpha
    if (pusher) {
        const VayMetric<float> vm{mm.alpha, mm.g_rr, mm.g_rp, mm.g_tt, mm.g_pp, mm.gi_rr, mm.gi_rp, mm.gi_tt,
                                  mm.gi_pp, mm.sqrtg};
        vay_step<float>(vm, qm, dt, D, B, u);
    } else {
        boris32<float>(mm, qm, dt, D, B, u);
    }
}

// The push of one particle of the near-horizon island with the native FP64
// metric and its derivatives (island_arith = 1).  o2 is the offset from the
// row's lower edge (stencils and window); in the last row (pole) the
// particle's theta offset is q = (pi - theta) / dtheta, stored with FP32's
// relative precision, and the trapezoid integrates q there (dq/dt =
// -X^theta / dtheta): on return q (pole) or o2 hold the end point's offset in
// that row's variable
template <int PUSHER>
__device__ __forceinline__ void push_island_fp64(const Push32Args &A, int i, int j, float &o1, float &o2, float u[3],
                                                 int sp, float &dphi, bool pole, float &q)
{
    const GridDev &g = A.g;
    const float rcf = (float)A.rcol[i + NG];
    const float d0 = rcf * expm1_cell(o1 * A.dx1f, A.dx1f);  // r - r_i
    // metric at x^n, shared by the Boris step and the first right-hand side
    const double am = g.a, r0 = A.rcol[i + NG] + (double)d0;
    double s0, c0;
    if (pole)
        sincos((double)g.nth * g.dth - (double)q * g.dth, &s0, &c0);
    else
        sincos(((double)j + (double)o2) * g.dth, &s0, &c0);
    KSGeo<double> m;
    ks_geo_sc<double>(am, r0, s0, c0, m);
    if ((A.boris_mask >> sp) & 1u) {
        float Dv[3], Bv[3];
        gather_fields32(A, i, j, o1, o2, Dv, Bv);
        boris_geo<double>(m, am, r0, s0, A.qm[sp], A.dt, Dv, Bv, u, PUSHER);
    }
    const float eps = ((A.massive_mask >> sp) & 1u) ? 1.0f : 0.0f;
    const float dt = A.dt, h = 0.5f * dt;
    const float idth = A.idthf;
    RhsT<float> f0, ft;
    geo_rhs_m<double, float>(m, eps, u[0], u[1], u[2], f0);
    f0.xt *= idth;
    // the theta offset integrated: o2 (X^theta / dtheta), or q in the pole
    // row (-X^theta / dtheta); sg is the sign and t0 the start value
    const float sg = pole ? -1.0f : 1.0f, t0 = pole ? q : o2;
    float a1 = d0 + dt * f0.xr, a2 = t0 + sg * dt * f0.xt, ap = dt * f0.xp;
    float b1 = u[0] + dt * f0.ur, b2 = u[1] + dt * f0.ut;
    for (int it = 0; it < A.n_iter; ++it) {
        // metric at the iterate: theta = theta^n + sg (a2 - t0) dtheta
        double s, c;
        const double d = sg * ((double)a2 - (double)t0) * g.dth;
        if (fabs(d) <= 0.05)
            sincos_shift<double>(s0, c0, d, s, c);
        else
            sincos(((double)j + (double)o2) * g.dth + d, &s, &c);
        const double ri = A.rcol[i + NG] + (double)a1;
        KSGeo<double> mi;
        ks_geo_sc<double>(am, ri, s, c, mi);
        geo_rhs_m<double, float>(mi, eps, b1, b2, u[2], ft);
        ft.xt *= idth;
        float n1 = d0 + h * (ft.xr + f0.xr), n2 = t0 + sg * h * (ft.xt + f0.xt);
        float nb1 = u[0] + h * (ft.ur + f0.ur), nb2 = u[1] + h * (ft.ut + f0.ut);
        ap = h * (ft.xp + f0.xp);
        bool done = false;
        if (A.use_tol) {
            // convergence test of the implicit iteration: change of the
            // iterate in r relative to r_i, in theta in radians (the same
            // relative length, r dtheta / r) and in u relative to max(1,
            // |u|).  The
            // difference of two floats within a factor 2 of each other is
            // exact in FP32 (Sterbenz's lemma), so for converging iterates
            // these differences are the FP64 ones; only the thresholds are
            // rounded to FP32.
            const float t = A.tolf;
            done = fabsf(n1 - a1) < t * rcf && fabsf(n2 - a2) < A.tol_o2 &&
                   fabsf(nb1 - b1) < t * fmaxf(1.0f, fabsf(nb1)) && fabsf(nb2 - b2) < t * fmaxf(1.0f, fabsf(nb2));
        }
        a1 = n1;
        a2 = n2;
        b1 = nb1;
        b2 = nb2;
        if (done) break;
    }
    o1 = log1p_cell(__fdividef(a1, rcf)) * A.idx1f;  // back to the logical offset
    if (pole)
        q = a2;
    else
        o2 = a2;
    u[0] = b1;
    u[1] = b2;
    dphi = ap;
}

// generalized Boris step in FP32 from the point quantities at x^n: the lower
// metric gamma_rr = 1 + z, gamma_thth = rho^2, gamma_rph = -a sin^2 (1 + z),
// gamma_phph = Sigma sin^2 / rho^2 with Sigma = (a^2 + r^2) rho^2 + 2 r a^2
// sin^2 (the same Sigma as (a^2 + r^2)^2 - a^2 Delta sin^2, without its
// cancellation), so gamma_phph = sin^2 (a^2 + r^2 + z a^2 sin^2); the upper
// metric of App. A and sqrt(gamma) = rho^2 sin sqrt(1 + z) = rho^2 sin (1 + z) alpha
__device__ __forceinline__ void boris_pt32(const Pt32 &m, float a, float a2, float qm, float dt, const float D[3],
                                           const float B[3], float u[3], int pusher)
{
    KSPoint<float> mm;
    mm.alpha = m.al;
    mm.g_rr = m.opz;
    mm.g_tt = m.rho2;
    mm.g_pp = m.s2 * fmaf(m.z, a2 * m.s2, m.ar2);
    mm.g_rp = -a * m.s2 * m.opz;
    mm.gi_rr = fmaf(m.ar2, m.ir, -m.beta);
    mm.gi_rp = a * m.ir;
    mm.gi_tt = m.ir;
    mm.gi_pp = m.ir * m.is2;
    mm.sqrtg = m.rho2 * m.s * m.opz * m.al;
    if (pusher) {
        const VayMetric<float> vm{mm.alpha, mm.g_rr, mm.g_rp, mm.g_tt, mm.g_pp, mm.gi_rr, mm.gi_rp, mm.gi_tt,
                                  mm.gi_pp, mm.sqrtg};
        vay_step<float>(vm, qm, dt, D, B, u);
    } else {
        boris32<float>(mm, qm, dt, D, B, u);
    }
}

// The push of one particle in FP32 (cells at or beyond fp64_radius): the
// point quantities at x^n serve the Boris step and the first right-hand
// side; sin and cos at the iterates from those at theta^n by the short
// series of sincos_shift (|shift| <= one cell).  Offsets and the pole row as
// in push_island_fp64; here sin, cos are those of theta itself (in the pole row cos
// theta = -cos theta' from the table of theta' = pi - theta), and the shift of
// theta per unit change of the integrated offset is +dtheta, or -dtheta in the
// pole row.
template <int PUSHER>
__device__ __forceinline__ void push_fp32(const Push32Args &A, int i, int j, float &o1, float &o2, float u[3], int sp,
                                          float &dphi, bool pole, float &q)
{
    const float2 rc2 = __ldg(reinterpret_cast<const float2 *>(A.rcol2) + i + NG);
    const float rcf = __fadd_rn(rc2.x, rc2.y);
    const float d0 = rcf * expm1_cell(o1 * A.dx1f, A.dx1f);  // r - r_i
    const float a = A.af;
    const float t0 = pole ? q : o2;  // the integrated theta offset at x^n
    const float4 sc = __ldg(reinterpret_cast<const float4 *>(A.rowsc) + (pole ? 0 : j));
    float s0, c0;
    sincos_shift<float>(sc.x, sc.z, t0 * A.dthf, s0, c0);
    if (pole) c0 = -c0;
    const Pt32 m0 = point32(A.a2f, A.m2a2f, rcf + d0, s0, c0);
    if ((A.boris_mask >> sp) & 1u) {
        float Dv[3], Bv[3];
        gather_fields32(A, i, j, o1, o2, Dv, Bv);
        boris_pt32(m0, a, A.a2f, A.qm[sp], A.dt, Dv, Bv, u, PUSHER);
    }
    const float eps = ((A.massive_mask >> sp) & 1u) ? 1.0f : 0.0f;
    const float dt = A.dt, h = 0.5f * dt;
    const float up = u[2], aup = a * up;
    RhsT<float> f0, ft;
    rhs32(m0, a, eps, u[0], u[1], up, aup, f0);
    // d(offset)/dt = sth X^theta; d theta = dsg d(offset)
    const float sth = pole ? -A.idthf : A.idthf, dsg = pole ? -A.dthf : A.dthf;
    const float hsth = h * sth;
    float a1 = fmaf(dt, f0.xr, d0), a2 = fmaf(dt * sth, f0.xt, t0);
    float b1 = fmaf(dt, f0.ur, u[0]), b2 = fmaf(dt, f0.ut, u[1]);
    float xpl = f0.xp;  // X^phi at the last evaluated iterate
    const float trc = A.tolf * rcf;
    for (int it = 0; it < A.n_iter; ++it) {
        const float d = (a2 - t0) * dsg;  // theta - theta^n
        float s, c;
        if (fabsf(d) <= 0.05f) {
            sincos_shift<float>(s0, c0, d, s, c);
        } else if (pole) {
            sincosf(t0 * A.dthf - d, &s, &c);  // theta' = pi - theta
            c = -c;
        } else {
            sincosf(((float)j + t0) * A.dthf + d, &s, &c);
        }
        const Pt32 mi = point32(A.a2f, A.m2a2f, rcf + a1, s, c);
        rhs32(mi, a, eps, b1, b2, up, aup, ft);
        xpl = ft.xp;
        const float n1 = fmaf(h, ft.xr + f0.xr, d0), n2 = fmaf(hsth, ft.xt + f0.xt, t0);
        const float nb1 = fmaf(h, ft.ur + f0.ur, u[0]), nb2 = fmaf(h, ft.ut + f0.ut, u[1]);
        bool done = false;
        if (A.use_tol) {
            // the convergence test of push_island_fp64: change of the iterate in r
            // relative to r_i, in theta in radians, in u relative to max(1, |u|)
            const float t = A.tolf;
            done = fabsf(n1 - a1) < trc && fabsf(n2 - a2) < A.tol_o2 && fabsf(nb1 - b1) < t * fmaxf(1.0f, fabsf(nb1)) &&
                   fabsf(nb2 - b2) < t * fmaxf(1.0f, fabsf(nb2));
        }
        a1 = n1;
        a2 = n2;
        b1 = nb1;
        b2 = nb2;
        if (done) break;
    }
    o1 = log1p_cell(__fdividef(a1, rcf)) * A.idx1f;  // back to the logical offset
    if (pole)
        q = a2;
    else
        o2 = a2;
    u[0] = b1;
    u[1] = b2;
    dphi = h * (xpl + f0.xp);  // dt X^phi(x^n) without correctors
}

// The island's point quantities in double-FP32 pairs: alpha, beta, gamma^ij,
// rho^2, 1/rho^2, 1 + z (and sin^2, 1/sin^2, a^2 + r^2, sin cos) in pairs,
// rounded to FP32 for the right-hand side; E = d_theta rho^2 / rho^2 in FP32
// from the rounded values (a derivative: force terms only).  The pairs the
// Boris step's lower metric reuses go to *keep.
struct IslandPt {
    df alpha, ir, opz, rho2, s2, ar2, z;
};

__device__ __forceinline__ void point_island(const df &a, const df &a2, float m2a2f, const df &r, const df &s,
                                             const df &c, Pt32 &m, GUp32 &gu, IslandPt *keep)
{
    const df r2 = r * r;
    const df rho2 = r2 + a2 * (c * c);
    const df ir = rcp_t(rho2);
    const df z = scale2(r, 2.0f) * ir;
    const df opz = add_f(z, 1.0f);
    const df iopz = rcp_t(opz);
    const df alpha = sqrt_t(iopz);
    const df beta = z * iopz;
    const df s2 = s * s;
    const df is2 = rcp_t(s2);
    const df ar2 = a2 + r2;
    m.s = (float)s;
    m.rho2 = (float)rho2;
    m.ir = (float)ir;
    m.z = (float)z;
    m.opz = (float)opz;
    m.al = (float)alpha;
    m.iopz = (float)iopz;
    m.beta = (float)beta;
    m.s2 = (float)s2;
    m.is2 = (float)is2;
    m.ar2 = (float)ar2;
    m.cs = (float)(c * s);
    m.E = m2a2f * m.cs * m.ir;
    gu.rr = (float)(ar2 * ir - beta);
    gu.rp = (float)(a * ir);
    gu.tt = m.ir;
    gu.pp = (float)(ir * is2);
    if (keep) {
        keep->alpha = alpha;
        keep->ir = ir;
        keep->opz = opz;
        keep->rho2 = rho2;
        keep->s2 = s2;
        keep->ar2 = ar2;
        keep->z = z;
    }
}

// the Boris step of an island particle: the lower metric from the pairs,
// gamma_phph = sin^2 (a^2 + r^2 + z a^2 sin^2) (Sigma without cancellation),
// gamma_rph = -a sin^2 (1 + z), sqrt(gamma) = rho^2 sin (1 + z) alpha
template <int PUSHER>
__device__ __forceinline__ void boris_island_pt(const Pt32 &m, const GUp32 &gu, const IslandPt &k, const df &a,
                                                const df &a2, const df &s, float qm, float dt, const float D[3],
                                                const float B[3], float u[3])
{
    KSPoint<float> mm;
    mm.alpha = m.al;
    mm.g_rr = m.opz;
    mm.g_tt = m.rho2;
    mm.g_pp = (float)(k.s2 * (k.ar2 + k.z * (a2 * k.s2)));
    mm.g_rp = (float)(-(a * k.s2 * k.opz));
    mm.gi_rr = gu.rr;
    mm.gi_rp = gu.rp;
    mm.gi_tt = gu.tt;
    mm.gi_pp = gu.pp;
    mm.sqrtg = (float)(k.rho2 * s * k.opz * k.alpha);
    if (PUSHER) {
        const VayMetric<float> vm{mm.alpha, mm.g_rr, mm.g_rp, mm.g_tt, mm.g_pp, mm.gi_rr, mm.gi_rp, mm.gi_tt,
                                  mm.gi_pp, mm.sqrtg};
        vay_step<float>(vm, qm, dt, D, B, u);
    } else {
        boris32<float>(mm, qm, dt, D, B, u);
    }
}

// The push of one particle of the near-horizon island with the metric in
// double-FP32 pairs: the steps of push_fp32 with the point quantities and
// gamma^ij from point_island (r as the pair r_i + (r - r_i), sin and cos of
// theta in pairs from the row table shifted by the offset), the right-hand
// sides by rhs32g.
template <int PUSHER>
__device__ __forceinline__ void push_island_df(const Push32Args &A, int i, int j, float &o1, float &o2, float u[3],
                                               int sp, float &dphi, bool pole, float &q)
{
    const float2 rc2 = __ldg(reinterpret_cast<const float2 *>(A.rcol2) + i + NG);
    const df rc(rc2.x, rc2.y);
    const float rcf = __fadd_rn(rc2.x, rc2.y);
    const float d0 = rcf * expm1_cell(o1 * A.dx1f, A.dx1f);  // r - r_i
    const float t0 = pole ? q : o2;
    const float4 sc = __ldg(reinterpret_cast<const float4 *>(A.rowsc) + (pole ? 0 : j));
    df s0, c0;
    sincos_shift_df(df(sc.x, sc.y), df(sc.z, sc.w), mul(A.dth_df, t0), s0, c0);
    if (pole) c0 = -c0;
    Pt32 m0;
    GUp32 g0;
    IslandPt keep;
    point_island(A.a_df, A.a2_df, A.m2a2f, add_f(rc, d0), s0, c0, m0, g0, &keep);
    if ((A.boris_mask >> sp) & 1u) {
        float Dv[3], Bv[3];
        gather_fields32(A, i, j, o1, o2, Dv, Bv);
        boris_island_pt<PUSHER>(m0, g0, keep, A.a_df, A.a2_df, s0, A.qm[sp], A.dt, Dv, Bv, u);
    }
    const float eps = ((A.massive_mask >> sp) & 1u) ? 1.0f : 0.0f;
    const float dt = A.dt, h = 0.5f * dt;
    const float up = u[2];
    RhsT<float> f0, ft;
    rhs32g(m0, g0, eps, u[0], u[1], up, f0);
    const float sth = pole ? -A.idthf : A.idthf;
    const df dsg = pole ? -A.dth_df : A.dth_df;
    const float hsth = h * sth;
    float a1 = fmaf(dt, f0.xr, d0), a2 = fmaf(dt * sth, f0.xt, t0);
    float b1 = fmaf(dt, f0.ur, u[0]), b2 = fmaf(dt, f0.ut, u[1]);
    float xpl = f0.xp;
    const float trc = A.tolf * rcf;
    for (int it = 0; it < A.n_iter; ++it) {
        const df d = two_sum(a2, -t0) * dsg;  // theta - theta^n
        df s, c;
        if (fabs_hi(d) <= 0.1f) {
            sincos_shift_df(s0, c0, d, s, c);
        } else if (pole) {
            sincos_t(mul(A.dth_df, t0) - d, &s, &c);  // theta' = pi - theta
            c = -c;
        } else {
            sincos_t(df(j) * A.dth_df + mul(A.dth_df, t0) + d, &s, &c);
        }
        Pt32 mi;
        GUp32 gi;
        point_island(A.a_df, A.a2_df, A.m2a2f, add_f(rc, a1), s, c, mi, gi, nullptr);
        rhs32g(mi, gi, eps, b1, b2, up, ft);
        xpl = ft.xp;
        const float n1 = fmaf(h, ft.xr + f0.xr, d0), n2 = fmaf(hsth, ft.xt + f0.xt, t0);
        const float nb1 = fmaf(h, ft.ur + f0.ur, u[0]), nb2 = fmaf(h, ft.ut + f0.ut, u[1]);
        bool done = false;
        if (A.use_tol) {
            const float t = A.tolf;
            done = fabsf(n1 - a1) < trc && fabsf(n2 - a2) < A.tol_o2 && fabsf(nb1 - b1) < t * fmaxf(1.0f, fabsf(nb1)) &&
                   fabsf(nb2 - b2) < t * fmaxf(1.0f, fabsf(nb2));
        }
        a1 = n1;
        a2 = n2;
        b1 = nb1;
        b2 = nb2;
        if (done) break;
    }
    o1 = log1p_cell(__fdividef(a1, rcf)) * A.idx1f;
    if (pole)
        q = a2;
    else
        o2 = a2;
    u[0] = b1;
    u[1] = b2;
    dphi = h * (xpl + f0.xp);
}

// resident 256-thread blocks per SM the register allocation is sized for
#ifndef GRPIC_PUSH32_MINB
#define GRPIC_PUSH32_MINB 4
#endif

// PUSHER: 0 generalized Boris, 1 Vay in the FIDO frame; IX: the slot index
// type (uint32_t while the capacity is below 2^31, int64_t beyond)
// slots per thread: a block of 256 threads takes GRPIC_PUSH32_PPT consecutive
// runs of 256 slots in turn (the per-thread setup is paid once for them)
#ifndef GRPIC_PUSH32_PPT
#define GRPIC_PUSH32_PPT 8
#endif

// one slot of the push (all 32 lanes of a warp call it: the deposit and the
// counts are warp collectives)
template <int PUSHER, typename IX>
__device__ __forceinline__ void push_slot(const Push32Args &A, const IX p, const IX nx, const bool permuted)
{
    const GridDev &g = A.g;
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int ncell = g.nr * g.nth;

    bool live = false;
    uint32_t tag = DEAD;
    int i = 0, j = 0, cellk = 0;
    float o1 = 0, o2 = 0, x2in = 0, u[3] = {0, 0, 0};
    if (p < nx) {
        const IX src = permuted ? (IX)A.perm[p] : p;
        tag = A.in_tag[src];
        if (!(tag & DEAD)) {
            cellk = A.in_cell[src];
            o1 = A.in_o1[src];
            o2 = x2in = A.in_o2[src];
            u[0] = A.in_u1[src];
            u[1] = A.in_u2[src];
            u[2] = A.in_u3[src];
            bool ok = cellk >= 0 && cellk < ncell && o1 >= 0.0f && o1 <= 1.0f && o2 >= 0.0f && o2 <= 1.0f &&
                      isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
            if (ok) {
                live = true;
                // cellk / n_r as a multiply-high by ceil(2^64 / n_r): exact
                // for cellk < 2^31 (the error term stays below 2^-33)
                j = (int)__umul64hi((unsigned long long)cellk, A.nr_recip);
                i = cellk - j * g.nr;
                // the last row stores q = (pi - theta) / dtheta; its offset
                // from the lower edge for the stencils and the window
                if (j == g.nth - 1) o2 = 1.0f - x2in;
            } else {
                bool fin = isfinite(o1) && isfinite(o2) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
                set_status(A.status, fin ? GRPIC_ERANGE : GRPIC_ENAN);
                tag |= DEAD;
            }
        }
    }

    bool dep = false, moved = false;
    float wa1 = 0, wa2 = 0, wb1 = 0, wb2 = 0, wq = 0, wphi = 0;  // window inputs (kept for regrouping)
    int key = -1, ni = i, nj = j;
    float n1 = o1, n2 = o2, x2out = x2in;
    if (live) {
        int sp = tag & 3u;
        float dphi = 0.0f;
        const bool pole = j == g.nth - 1;
        float q = x2in;
        // FP64 island: cells whose inner edge r_i lies below fp64_radius
        if (i >= A.i64)
            push_fp32<PUSHER>(A, i, j, n1, n2, u, sp, dphi, pole, q);
        else if (A.island_fp64)
            push_island_fp64<PUSHER>(A, i, j, n1, n2, u, sp, dphi, pole, q);
        else
            push_island_df<PUSHER>(A, i, j, n1, n2, u, sp, dphi, pole, q);
        // axis reflection (theta = 0 is o2 = 0 of row 0, theta = pi is q = 0
        // of the last row); the end point relative to the start row's lower edge
        if (j == 0 && n2 < 0.0f) { n2 = -n2; u[1] = -u[1]; }
        if (pole) {
            if (q < 0.0f) { q = -q; u[1] = -u[1]; }
            n2 = 1.0f - q;
        }
        bool finite = isfinite(n1) && isfinite(n2) && isfinite(u[0]) && isfinite(u[1]) && isfinite(dphi);
        if (!finite) {
            set_status(A.status, GRPIC_ENAN);
            tag |= DEAD;
        } else {
            int di = (int)floorf(n1), dj = (int)floorf(n2);
            if (dj > 0 && j + dj > g.nth - 1) dj = g.nth - 1 - j;  // theta = pi exactly stays in the last row
            if (di < -1 || di > 1 || dj < -1 || dj > 1) {
                set_status(A.status, GRPIC_ERANGE);
                tag |= DEAD;
            } else {
                // inputs of the Esirkepov window (columns i-1..i+2, rows j-1..j+2);
                // the end point (n1, n2) is relative to the start cell
                wq = A.qw[sp];
                wa1 = o1;
                wa2 = o2;
                wb1 = n1;
                wb2 = n2;
                wphi = dphi;
                dep = true;
                moved = true;
                ni = i + di;
                nj = j + dj;
                n1 -= (float)di;
                n2 -= (float)dj;
                if (n1 >= 1.0f) n1 = 0x1.fffffep-1f;  // rounding of the re-centring
                if (n1 < 0.0f) n1 = 0.0f;
                if (n2 > 1.0f) n2 = 1.0f;
                if (n2 < 0.0f) n2 = 0.0f;
                // the stored offset: q in the last row (kept as integrated when
                // the particle stays there), the lower-edge offset elsewhere
                if (nj == g.nth - 1)
                    x2out = (pole && dj == 0) ? fminf(fmaxf(q, 0.0f), 1.0f) : 1.0f - n2;
                else
                    x2out = n2;
                if (ni < 0 || ni >= g.nr) tag |= DEAD;  // left [r_in, r_out)
                key = (tag & DEAD) ? ncell : nj * g.nr + ni;
            }
        }
    }
    if (p < nx) {
        if (moved || permuted) {
            A.cell[p] = nj * g.nr + ni;
            A.o1[p] = n1;
            A.o2[p] = x2out;
            A.u1[p] = u[0];
            A.u2[p] = u[1];
            A.u3[p] = u[2];
        }
        if (tag & DEAD) key = ncell;
        A.tag[p] = tag;
        A.keys[p] = key;
    } else if (permuted && p < (IX)A.n) {
        A.tag[p] = DEAD;  // past the live slots of the permuted order
    }

    if (A.cnt9) {
        // old cell = start cell (the slot's segment of the permuted order);
        // lanes match on cell * 9 + direction (32-bit: the cells of one warp
        // lie far closer together than 2^32 / 9)
        const bool counted = p < nx && moved && !(tag & DEAD);
        const int dir = (nj - j + 1) * 3 + (ni - i + 1);
        const unsigned mk = counted ? (unsigned)cellk * 9u + (unsigned)dir : 0xffffffffu;
        const unsigned peers = __match_any_sync(FULL, mk);
        if (counted && lane == __ffs(peers) - 1) atomicAdd(A.cnt9 + (int64_t)dir * ncell + cellk, (int)__popc(peers));
    }

    if (A.histogram) {
        int hk = (p < nx) ? key : -1;
        unsigned peers = __match_any_sync(FULL, hk);
        if (hk >= 0 && lane == __ffs(peers) - 1) atomicAdd(A.count + hk, __popc(peers));
    }

    // ---- deposit: lanes grouped by start cell, each group reduce-scattered --
    deposit_warp_split<float, 3>(dep, i, j, g.nr, wa1, wa2, wb1, wb2, wq * A.m_i2dt, wq * A.idt, wphi, lane, g.nth,
                                 NG, A.ldi, A.J0,
                                 A.J1, A.J2);
}

template <int PUSHER, typename IX>
__global__ void __launch_bounds__(256, GRPIC_PUSH32_MINB) push32_kernel(Push32Args A)
{
    const bool permuted = A.perm != nullptr;
    int64_t n = permuted ? (int64_t)*A.live : (A.d_count ? *A.d_count : A.n);
    if (n > A.n) n = A.n;
    const IX nx = (IX)n;
    const IX p0 = (IX)blockIdx.x * (blockDim.x * GRPIC_PUSH32_PPT) + threadIdx.x;
    if (permuted && p0 == 0 && A.count_out) *A.count_out = n;
#pragma unroll 1
    for (int k = 0; k < GRPIC_PUSH32_PPT; ++k) push_slot<PUSHER, IX>(A, p0 + (IX)(k * blockDim.x), nx, permuted);
}

// The stencil quads of the six field components, interleaved by point (the
// components of one stencil point share 96 bytes): for the stencil whose
// first row is js (-1 .. n_theta - 1) and first column col,
//   Q[6 ((js + 1) ld + col) + c] = (F_c[r0][col], F_c[r0][col + 1], F_c[r1][col], F_c[r1][col + 1])
// with r0 = js, r1 = js + 1.  The components at half-integer theta (D^theta,
// odd across the axis; B^r and B^phi, even) have rows 0 .. n_theta - 1: a row
// beyond them is its mirror across the axis (-1 -> 0, n_theta -> n_theta - 1)
// times the parity.  Entries no stencil reads (the last column, row js = -1
// of the integer-theta components) are zero.  A parity of -1 commutes with
// rounding, so the gathers equal those from the arrays themselves bit for bit.
struct Quad32Args {
    const float *F[6];
    float4 *Q;
    int nth, ld;
    // zeroed on the way (the push deposits into J and counts into cnt9):
    // J[c] over the same (nth+1) x ld points, cnt9 (9 x nr x nth) if given
    float *J[3];
    int32_t *cnt9;
    int nr;
};

// One block row per stencil row js + 1 (blockIdx.y); along x the row's work
// elements e: quad element 6 col + c (consecutive lanes store consecutive
// 16-byte quads), the zeroed J entries k ld + col, the zeroed counts d n_r + i.
__global__ void quad32_kernel(Quad32Args A)
{
    const int qr = blockIdx.y;  // js + 1
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (qr > A.nth) return;
    const int ld = A.ld;
    if (e < 6 * ld) {
        const int col = e / 6, c = e - 6 * col;
        const int js = qr - 1;
        const bool half_t = (c & 1) != 0;  // D^theta (1), B^r (3), B^phi (5)
        const float par = c == 1 ? -1.0f : 1.0f;
        int r0 = js, r1 = js + 1;
        float p0 = 1.0f, p1 = 1.0f;
        if (half_t) {
            if (r0 < 0) { r0 = -1 - r0; p0 = par; }
            if (r1 > A.nth - 1) { r1 = 2 * A.nth - 1 - r1; p1 = par; }
        }
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (r0 >= 0 && col + 1 < ld) {
            // by selects: a run-time index into the parameter array would
            // copy the array to local memory in every thread
            const float *F = c < 3 ? (c == 0 ? A.F[0] : (c == 1 ? A.F[1] : A.F[2]))
                                   : (c == 3 ? A.F[3] : (c == 4 ? A.F[4] : A.F[5]));
            const float *a = F + (size_t)r0 * ld + col;
            const float *b = F + (size_t)r1 * ld + col;
            v = make_float4(p0 * a[0], p0 * a[1], p1 * b[0], p1 * b[1]);
        }
        A.Q[(size_t)qr * 6 * ld + e] = v;
    }
    if (A.J[0] && e < 3 * ld) {
        const int k = e / ld;
        float *J = k == 0 ? A.J[0] : (k == 1 ? A.J[1] : A.J[2]);
        J[(size_t)qr * ld + (e - k * ld)] = 0.0f;
    }
    if (A.cnt9 && qr < A.nth && e < 9 * A.nr) {
        const int d = e / A.nr;
        A.cnt9[(size_t)d * A.nr * A.nth + (size_t)qr * A.nr + (e - d * A.nr)] = 0;
    }
}

}  // namespace

cudaError_t launch_quad32(grpic_ctx *ctx, grpic_fields *f, bool zero_j, int32_t *zero_cnt9, cudaStream_t s)
{
    if (!ctx->q32 || ctx->fscratch_ld != f->ld || f->ld < ctx->g.nr) return cudaErrorInvalidValue;
    Quad32Args A;
    for (int c = 0; c < 3; ++c) A.J[c] = zero_j ? (float *)f->J[c] : nullptr;
    A.cnt9 = zero_cnt9;
    A.nr = ctx->g.nr;
    for (int c = 0; c < 3; ++c) {
        A.F[c] = (const float *)f->D[c];
        A.F[c + 3] = (const float *)f->B[c];
    }
    A.Q = static_cast<float4 *>(ctx->q32);
    A.nth = ctx->g.nth;
    A.ld = (int)f->ld;
    const int64_t w = std::max<int64_t>(6 * f->ld, 9 * (int64_t)ctx->g.nr);  // work elements per row
    const dim3 grid((unsigned)((w + 255) / 256), (unsigned)(ctx->g.nth + 1));
    quad32_kernel<<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_push32(grpic_ctx *ctx, const grpic_particles *in, grpic_particles *p, const int32_t *perm,
                          const int32_t *live, int32_t *cnt9, grpic_fields *f, bool histogram, cudaStream_t s,
                          int64_t slot0)
{
    Push32Args A;
    A.g = ctx->g;
    A.dt = (float)ctx->prm.dt;
    A.idt = (float)(1.0 / ctx->prm.dt);
    A.m_i2dt = (float)(-0.5 / ctx->prm.dt);
    A.n_iter = ctx->prm.n_push_iter;
    A.tolf = (float)ctx->prm.push_tol;
    A.tol_o2 = (float)(ctx->prm.push_tol / ctx->g.dth);
    A.massive_mask = A.boris_mask = 0u;
    for (int k = 0; k < 4; ++k) {
        A.qm[k] = (float)ctx->prm.q_over_m[k];
        A.qw[k] = (float)ctx->prm.q_weight[k];
        A.massive[k] = ctx->prm.massive[k];
        if (A.massive[k]) A.massive_mask |= 1u << k;
        if (A.massive[k] && A.qm[k] != 0.0f) A.boris_mask |= 1u << k;
    }
    A.r64 = ctx->prm.fp64_radius;
    A.island_fp64 = ctx->prm.island_arith == 1 ? 1 : 0;
    A.use_tol = ctx->prm.push_tol > 0.0 ? 1 : 0;
    A.af = (float)ctx->g.a;
    A.a2f = (float)(ctx->g.a * ctx->g.a);
    A.m2a2f = (float)(-2.0 * ctx->g.a * ctx->g.a);
    A.dthf = (float)ctx->g.dth;
    A.idthf = (float)(1.0 / ctx->g.dth);
    A.dx1f = (float)ctx->g.dx1;
    A.idx1f = (float)(1.0 / ctx->g.dx1);
    A.a_df = df_const(ctx->g.a);
    A.a2_df = df_const(ctx->g.a * ctx->g.a);
    A.dth_df = df_const(ctx->g.dth);
    A.rcol2 = ctx->rcol2;
    A.rowsc = ctx->rowsc;
    A.i64 = 0;
    if (A.r64 > 0.0)
        while (A.i64 < ctx->g.nr && ctx->g.r_in * std::exp(A.i64 * ctx->g.dx1) < A.r64) ++A.i64;
    A.n = p->n;
    A.d_count = p->d_count;
    A.cell = p->cell;
    A.o1 = (float *)p->x1;
    A.o2 = (float *)p->x2;
    A.u1 = (float *)p->u1;
    A.u2 = (float *)p->u2;
    A.u3 = (float *)p->u3;
    A.tag = p->tag;
    A.perm = perm;
    A.live = live;
    A.count_out = perm ? p->d_count : nullptr;
    A.cnt9 = perm ? cnt9 : nullptr;
    A.in_cell = in->cell;
    A.in_o1 = (const float *)in->x1;
    A.in_o2 = (const float *)in->x2;
    A.in_u1 = (const float *)in->u1;
    A.in_u2 = (const float *)in->u2;
    A.in_u3 = (const float *)in->u3;
    A.in_tag = in->tag;
    if (!ctx->q32 || ctx->fscratch_ld != f->ld) return cudaErrorInvalidValue;  // launch_quad32 comes first
    A.Q = static_cast<const float4 *>(ctx->q32);
    A.J0 = (float *)f->J[0];
    A.J1 = (float *)f->J[1];
    A.J2 = (float *)f->J[2];
    A.ld = f->ld;
    A.ldi = (int)f->ld;
    A.rcol = ctx->rcol;
    A.keys = ctx->d_keys + slot0;
    A.count = ctx->d_count;
    A.histogram = histogram ? 1 : 0;
    A.status = ctx->d_status;
    A.nr_recip = ~0ull / (unsigned long long)ctx->g.nr + 1ull;
    if (p->n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((p->n + 256 * GRPIC_PUSH32_PPT - 1) / (256 * GRPIC_PUSH32_PPT));
    const bool narrow = p->capacity < ((int64_t)1 << 31) - 256 * GRPIC_PUSH32_PPT;
    if (ctx->prm.pusher) {
        if (narrow)
            push32_kernel<1, uint32_t><<<blocks, 256, 0, s>>>(A);
        else
            push32_kernel<1, int64_t><<<blocks, 256, 0, s>>>(A);
    } else {
        if (narrow)
            push32_kernel<0, uint32_t><<<blocks, 256, 0, s>>>(A);
        else
            push32_kernel<0, int64_t><<<blocks, 256, 0, s>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace grpic
