// grpic_push64.cu -- FP64 particle push fused with the charge-conserving
// deposit (arXiv:2503.04558 Sec. 2.2-2.3, Fig. stepping).
//
// One thread per particle (structure of arrays, coalesced loads):
//   1. interpolate D^j, B^j at x^n, each from its own staggered lattice
//      (bilinear cloud-in-cell in logical coordinates);
//   2. one full generalized Boris step at fields n (Eqs. boris-plus-minus,
//      u0bar, boris-scheme), skipped for photons;
//   3. geodesic predictor + n_iter trapezoidal correctors (Eqs.
//      geodesic-predictor, geodesic-corrector) on (r, theta, phi, u_r, u_theta);
//      U_phi = 0 so u_phi is left untouched;
//   4. axis reflection, range / finiteness checks;
//   5. Esirkepov deposit of x^n -> x^{n+1} (Eq. esirkepov-decomp with a local
//      prefix sum, Eq. j-phi-deposit) into the integrated currents
//      J^r A_r, J^theta A_theta, J^phi dV.  With CIC weights the prefix sums
//      factor per dimension:  J^r A_r(k+1/2, l) = -qw/(2dt) P_r(k) (S1_t + S0_t)(l)
//      with P_r(k) = sum_{k'<=k} (S1_r - S0_r)(k'), and likewise for theta.
//      A warp whose particles all start in one cell (the usual case after the
//      sort) reduce-scatters its 4x4-window contributions over the lanes and
//      each lane adds at most two totals; otherwise each lane adds its own;
//   6. cell key of x^{n+1} (dead -> n_cells) and a warp-aggregated histogram
//      for the sort.
#include "grpic_internal.cuh"
#include "grpic_geo.cuh"
#include "grpic_window.cuh"
#include "grpic_vay.cuh"
#include "grpic_shape3.cuh"
#include "grpic_philox.cuh"

namespace grpic {
namespace {

struct Push64Args {
    GridDev g;
    double dt;
    double idt, m_i2dt;  // 1 / dt, -1 / (2 dt)
    int n_iter;
    double qm[4], qw[4];
    int massive[4];
    int64_t n;
    const int64_t *d_count;
    double *r, *th, *u1, *u2, *u3;
    uint32_t *tag;
    // read through a permutation (see the FP32 push): slot p's particle comes
    // from slot perm[p] of the input arrays; perm == nullptr: in place
    const int32_t *perm, *live;
    int64_t *count_out;
    int32_t *cnt9;  // with perm: counts of the next neighbour sort (see the FP32 push)
    const double *in_r, *in_th, *in_u1, *in_u2, *in_u3;
    const uint32_t *in_tag;
    const double *D0, *D1, *D2, *B0, *B1, *B2;
    double *J0, *J1, *J2;
    int64_t ld;
    int32_t *keys;
    int32_t *count;
    int histogram;
    int pusher;  // 0 generalized Boris, 1 Vay in the FIDO frame
    // 2D radiation: emission / conversion decisions per slot into spawn
    // (0, 1 photon, 2 pair), see grpic_rad.cu
    int radiation;
    double gamma_thr, eps_ph, pconv;
    uint64_t seed;
    int64_t step;
    int32_t *spawn;
    int *status;
    double *tape;  // the adjoint's record of the push (TAPE instantiation only)
    int64_t tape_ld;
};

using Rhs = RhsT<double>;
using Pt64 = PtT<double>;

// the right-hand side of Eq. particle-eom (without F_i) at a point: the
// point quantities and the part in u of grpic_geo.cuh's pointT / rhsT
__device__ __forceinline__ void geo_rhs_sc(double a, double a2, double m2a2, double eps, double r, double s, double c,
                                           double ur, double ut, double up, Rhs &f)
{
    const Pt64 m = pointT<double>(a2, m2a2, r, s, c);
    rhsT<double>(m, a, eps, ur, ut, up, a * up, f);
}

// the 3+1 metric at the point (App. A): gamma_rr = 1 + z, gamma_thth = rho^2,
// gamma_rph = -a sin^2 (1 + z), gamma_phph = Sigma sin^2 / rho^2 with Sigma =
// (a^2 + r^2) rho^2 + 2 r a^2 sin^2 (the same Sigma as (a^2 + r^2)^2 - a^2
// Delta sin^2, without its cancellation), so gamma_phph = sin^2 (a^2 + r^2 +
// z a^2 sin^2); sqrt(gamma) = rho^2 sin (1 + z) alpha
__device__ __forceinline__ void ks_point_pt(double a, double a2, const Pt64 &B, KS &m)
{
    m.alpha = B.al;
    m.beta = B.beta;
    m.g_rr = B.opz;
    m.g_tt = B.rho2;
    m.g_pp = B.s2 * fma(B.z, a2 * B.s2, B.ar2);
    m.g_rp = -a * B.s2 * B.opz;
    m.gi_rr = fma(B.ar2, B.ir, -B.beta);
    m.gi_rp = a * B.ir;
    m.gi_tt = B.ir;
    m.gi_pp = B.ir * B.is2;
    m.sqrtg = B.rho2 * B.s * B.opz * B.al;
}

// Generalized Boris step over dt at the particle (u covariant, D, B
// contravariant) with the point quantities at x^n
__device__ __forceinline__ void boris(double a, double a2, const Pt64 &Bm, double qm, double dt, const double D[3],
                                      const double B[3], double u[3])
{
    KS m;
    ks_point_pt(a, a2, Bm, m);
    double Dl0 = m.g_rr * D[0] + m.g_rp * D[2];
    double Dl1 = m.g_tt * D[1];
    double Dl2 = m.g_rp * D[0] + m.g_pp * D[2];
    double h = 0.5 * qm * m.alpha * dt;
    double um0 = u[0] + h * Dl0, um1 = u[1] + h * Dl1, um2 = u[2] + h * Dl2;
    // raised u^-
    double v0 = m.gi_rr * um0 + m.gi_rp * um2, v1 = m.gi_tt * um1, v2 = m.gi_rp * um0 + m.gi_pp * um2;
    double iu0b = m.alpha * rsqrt_fast(1.0 + um0 * v0 + um1 * v1 + um2 * v2);  // 1 / u0bar
    double kt = 0.5 * qm * dt * iu0b;
    double t0 = kt * B[0], t1 = kt * B[1], t2 = kt * B[2];
    double tt = t0 * (m.g_rr * t0 + m.g_rp * t2) + t1 * (m.g_tt * t1) + t2 * (m.g_rp * t0 + m.g_pp * t2);
    double ks = 2.0 * rcp_t(1.0 + tt);
    double s0 = ks * t0, s1 = ks * t1, s2 = ks * t2;
    double sg = m.sqrtg;
    // u~ = u^- + e_ijk v^j t^k
    double w0 = um0 + sg * (v1 * t2 - v2 * t1);
    double w1 = um1 + sg * (v2 * t0 - v0 * t2);
    double w2 = um2 + sg * (v0 * t1 - v1 * t0);
    double x0 = m.gi_rr * w0 + m.gi_rp * w2, x1 = m.gi_tt * w1, x2 = m.gi_rp * w0 + m.gi_pp * w2;
    // u^+ = u^- + e_ijk (raised u~)^j s^k, then the second electric half kick
    u[0] = um0 + sg * (x1 * s2 - x2 * s1) + h * Dl0;
    u[1] = um1 + sg * (x2 * s0 - x0 * s2) + h * Dl1;
    u[2] = um2 + sg * (x0 * s1 - x1 * s0) + h * Dl2;
}

// Vay's update in the FIDO frame with the metric at (r, theta)
__device__ __forceinline__ void vay(double a, double r, double th, double qm, double dt, const double D[3],
                                    const double B[3], double u[3])
{
    KS k;
    ks_point(a, r, th, k);
    VayMetric<double> m{k.alpha, k.g_rr, k.g_rp, k.g_tt, k.g_pp, k.gi_rr, k.gi_rp, k.gi_tt, k.gi_pp, k.sqrtg};
    vay_step<double>(m, qm, dt, D, B, u);
}

// bilinear weights on a lattice staggered by (sr, st) cells
struct Stencil {
    int c0, r0, r1;       // column of the lower corner, the two row indices
    double w00, w10, w01, w11;
    double p0, p1;        // parities of the two rows (reflection across the axis)
};

__device__ __forceinline__ void stencil(const GridDev &g, double x1, double x2, bool half_r, bool half_t, double par,
                                        Stencil &S)
{
    double xi = half_r ? x1 - 0.5 : x1;
    double fi = floor(xi);
    int i = (int)fi;
    double f = xi - fi;
    int j;
    double gfr;
    S.p0 = S.p1 = 1.0;
    if (half_t) {
        double eta = x2 - 0.5;
        double fj = floor(eta);
        j = (int)fj;
        gfr = eta - fj;
        // half-theta rows: -1 mirrors 0, nth mirrors nth-1
        S.r0 = j;
        S.r1 = j + 1;
        if (S.r0 < 0) { S.r0 = -1 - S.r0; S.p0 = par; }
        if (S.r1 > g.nth - 1) { S.r1 = 2 * g.nth - 1 - S.r1; S.p1 = par; }
    } else {
        double fj = floor(x2);
        j = (int)fj;
        if (j > g.nth - 1) j = g.nth - 1;
        gfr = x2 - j;
        S.r0 = j;
        S.r1 = j + 1;
    }
    S.c0 = i + NG;
    S.w00 = (1.0 - f) * (1.0 - gfr);
    S.w10 = f * (1.0 - gfr);
    S.w01 = (1.0 - f) * gfr;
    S.w11 = f * gfr;
}

__device__ __forceinline__ double gather(const double *__restrict__ F, int64_t ld, const Stencil &S)
{
    const double *a = F + (size_t)S.r0 * ld + S.c0;
    const double *b = F + (size_t)S.r1 * ld + S.c0;
    return S.p0 * (S.w00 * __ldg(a) + S.w10 * __ldg(a + 1)) + S.p1 * (S.w01 * __ldg(b) + S.w11 * __ldg(b + 1));
}


__device__ __forceinline__ int jcell(const GridDev &g, double x2)
{
    int j = (int)floor(x2);
    return j > g.nth - 1 ? g.nth - 1 : j;
}

// SHAPE 1: cloud in cell (bilinear interpolation, 4 x 4 window reduced across
// the warp); SHAPE 3: the cubic spline of grpic_shape3.cuh (4 x 4 taps,
// per-lane deposit of the 5 x 5 window).  TAPE: also write the adjoint's
// record of the push (CIC, no radiation)
template <int SHAPE, bool RAD, bool TAPE>
__global__ void __launch_bounds__(256) push64_kernel(Push64Args A)
{
    const GridDev &g = A.g;
    const bool permuted = A.perm != nullptr;
    int64_t n = permuted ? (int64_t)*A.live : (A.d_count ? *A.d_count : A.n);
    if (n > A.n) n = A.n;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int ncell = g.nr * g.nth;
    if (permuted && p == 0 && A.count_out) *A.count_out = n;

    bool live = false;
    uint32_t tag = DEAD;
    double r = 0, th = 0, u[3] = {0, 0, 0};
    if (p < n) {
        const int64_t src = permuted ? (int64_t)A.perm[p] : p;
        tag = A.in_tag[src];
        if (!(tag & DEAD)) {
            live = true;
            r = A.in_r[src];
            th = A.in_th[src];
            u[0] = A.in_u1[src];
            u[1] = A.in_u2[src];
            u[2] = A.in_u3[src];
        }
    }

    bool dep = false;
    int spawn = 0;
    double wa1 = 0.0, wa2 = 0.0, wb1 = 0.0, wb2 = 0.0, wq = 0.0, wphi = 0.0;  // window inputs (CIC)
    int i0 = 0, j0 = 0, key = -1;
    if (live) {
        // a state outside the domain (or non-finite) would index the fields out
        // of range: refuse it before any gather
        bool inside = isfinite(r) && isfinite(th) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) &&
                      r >= g.r_in && r < g.r_out && th >= 0.0 && th <= M_PI;
        if (!inside) {
            bool fin = isfinite(r) && isfinite(th) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
            set_status(A.status, fin ? GRPIC_ERANGE : GRPIC_ENAN);
            tag |= DEAD;
            live = false;
        }
    }
    if (live) {
        int sp = tag & 3u;
        double x1a = (log(r) - g.ln_rin) / g.dx1, x2a = th / g.dth;
        if (x1a >= (double)g.nr) x1a = nextafter((double)g.nr, 0.0);  // rounding just below r_out
        if (x1a < 0.0) x1a = 0.0;
        // sin, cos of theta^n: shared by the Boris step and the first
        // right-hand side, shifted for the corrector iterates
        double s0, c0;
        sincos(th, &s0, &c0);
        const double a2 = g.a * g.a, m2a2 = -2.0 * a2;
        const Pt64 B0 = pointT<double>(a2, m2a2, r, s0, c0);
        if (A.massive[sp] && A.qm[sp] != 0.0) {
            double Dv[3], Bv[3];
            if constexpr (SHAPE == 3) {
                gather3_fields(A.D0, A.D1, A.D2, A.B0, A.B1, A.B2, A.ld, g.nth, x1a, x2a, Dv, Bv);
            } else {
                Stencil Sh0, S0h, S00, Shh;
                stencil(g, x1a, x2a, true, false, 1.0, Sh0);   // D^r, B^theta
                stencil(g, x1a, x2a, false, true, -1.0, S0h);  // D^theta (odd across the axis)
                stencil(g, x1a, x2a, false, false, 1.0, S00);  // D^phi
                stencil(g, x1a, x2a, true, true, 1.0, Shh);    // B^phi
                Dv[0] = gather(A.D0, A.ld, Sh0);
                Dv[1] = gather(A.D1, A.ld, S0h);
                Dv[2] = gather(A.D2, A.ld, S00);
                Bv[1] = gather(A.B1, A.ld, Sh0);
                Bv[2] = gather(A.B2, A.ld, Shh);
                S0h.p0 = S0h.p1 = 1.0;  // B^r is even across the axis
                Bv[0] = gather(A.B0, A.ld, S0h);
            }
            if (A.pusher)
                vay(g.a, r, th, A.qm[sp], A.dt, Dv, Bv, u);
            else
                boris(g.a, a2, B0, A.qm[sp], A.dt, Dv, Bv, u);
        }
        // geodesic predictor-corrector (Sec. 2.2)
        double eps = A.massive[sp] ? 1.0 : 0.0;
        Rhs f0, ft;
        double *tape = TAPE ? A.tape + p : nullptr;
        const int64_t tl = A.tape_ld;
        if constexpr (TAPE) {
            tape[(TAPE_U + 0) * tl] = u[0];
            tape[(TAPE_U + 1) * tl] = u[1];
            tape[(TAPE_U + 2) * tl] = u[2];
            tape[TAPE_SC0 * tl] = s0;
            tape[(TAPE_SC0 + 1) * tl] = c0;
        }
        rhsT<double>(B0, g.a, eps, u[0], u[1], u[2], g.a * u[2], f0);
        double dt = A.dt;
        double rt = r + dt * f0.xr, tt = th + dt * f0.xt, pt = dt * f0.xp;
        double urt = u[0] + dt * f0.ur, utt = u[1] + dt * f0.ut;
        for (int it = 0; it < A.n_iter; ++it) {
            // theta of the iterate within 0.05 of theta^n (the usual case: one
            // step moves a particle less than two cells): the series of
            // sincos_shift, truncated below 1e-17
            double st, ct;
            const double dth = tt - th;
            if (fabs(dth) <= 0.05)
                sincos_shift<double>(s0, c0, dth, st, ct);
            else
                sincos(tt, &st, &ct);
            if constexpr (TAPE) {
                double *q = tape + (int64_t)(TAPE_IT + 6 * it) * tl;
                q[0] = rt;
                q[tl] = tt;
                q[2 * tl] = urt;
                q[3 * tl] = utt;
                q[4 * tl] = st;
                q[5 * tl] = ct;
            }
            geo_rhs_sc(g.a, a2, m2a2, eps, rt, st, ct, urt, utt, u[2], ft);
            double h = 0.5 * dt;
            rt = r + h * (ft.xr + f0.xr);
            tt = th + h * (ft.xt + f0.xt);
            pt = h * (ft.xp + f0.xp);
            urt = u[0] + h * (ft.ur + f0.ur);
            utt = u[1] + h * (ft.ut + f0.ut);
        }
        if constexpr (TAPE) {
            double *q = tape + (int64_t)tape_end(A.n_iter) * tl;
            q[0] = rt;
            q[tl] = tt;
            q[2 * tl] = urt;
            q[3 * tl] = utt;
            q[4 * tl] = pt;
        }
        // axis reflection
        if (tt < 0.0) { tt = -tt; utt = -utt; }
        if (tt > M_PI) { tt = 2.0 * M_PI - tt; utt = -utt; }
        bool finite = isfinite(rt) && isfinite(tt) && isfinite(pt) && isfinite(urt) && isfinite(utt) && rt > 0.0;
        if (!finite) {
            set_status(A.status, GRPIC_ENAN);
            tag |= DEAD;
            live = false;
        } else {
            double x1b = (log(rt) - g.ln_rin) / g.dx1, x2b = tt / g.dth;
            i0 = (int)floor(x1a);
            j0 = jcell(g, x2a);
            int di = (int)floor(x1b) - i0, dj = jcell(g, x2b) - j0;
            if (di < -1 || di > 1 || dj < -1 || dj > 1) {
                set_status(A.status, GRPIC_ERANGE);
                tag |= DEAD;
                live = false;
            } else {
                if constexpr (SHAPE == 3) {
                    deposit3(g.nr, g.nth, A.ld, A.J0, A.J1, A.J2, A.qw[tag & 3u], dt, x1a, x2a, x1b, x2b, pt);
                } else {
                    // inputs of the split window deposit, relative to the
                    // start cell (i0, j0): the start in [0, 1], the end in [-1, 2]
                    wq = A.qw[tag & 3u];
                    wa1 = x1a - i0;
                    wa2 = x2a - j0;
                    wb1 = x1b - i0;
                    wb2 = x2b - j0;
                    wphi = pt;
                }
                dep = true;
                r = rt;
                th = tt;
                u[0] = urt;
                u[1] = utt;
                if (rt < g.r_in || rt >= g.r_out) tag |= DEAD;
                // the column the next push will start from (it clamps x1 into [0, nr))
                int ib = (int)floor(x1b);
                ib = ib < 0 ? 0 : (ib > g.nr - 1 ? g.nr - 1 : ib);
                key = (tag & DEAD) ? ncell : (jcell(g, x2b) * g.nr + ib);
                if (RAD && !(tag & DEAD)) {
                    // at the new position: emission by a charged particle above
                    // gamma_thr, conversion of a photon above 2 m c^2; a photon
                    // draws first (the draw fails for all but ~tau dt of them,
                    // which then skip the metric: the same decision)
                    const bool charged = A.massive[sp] && A.qm[sp] != 0.0;
                    const bool drawn = !A.massive[sp] && uniform53(A.seed, (uint64_t)p, A.step, 1) < A.pconv;
                    if (charged || drawn) {
                        KS m;
                        ks_point(g.a, r, th, m);
                        const double uu = m.gi_rr * u[0] * u[0] + 2.0 * m.gi_rp * u[0] * u[2] +
                                          m.gi_tt * u[1] * u[1] + m.gi_pp * u[2] * u[2];
                        if (charged) {
                            const double G = sqrt(1.0 + uu), G2 = G - A.eps_ph;
                            if (G >= A.gamma_thr && G2 >= 1.0) {
                                const double f = sqrt(G2 * G2 - 1.0) / sqrt(uu);
                                u[0] *= f;
                                u[1] *= f;
                                u[2] *= f;
                                spawn = 1;
                            }
                        } else if (sqrt(uu) > 2.0) {
                            spawn = 2;
                            tag |= DEAD;
                            key = ncell;
                        }
                    }
                }
            }
        }
    }
    if (RAD && p < n) A.spawn[p] = spawn;
    if (p < n) {
        if (dep || permuted) {
            A.r[p] = r;
            A.th[p] = th;
            A.u1[p] = u[0];
            A.u2[p] = u[1];
            A.u3[p] = u[2];
        }
        if (tag & DEAD) key = ncell;
        A.tag[p] = tag;
        A.keys[p] = key;
    } else if (permuted && p < A.n) {
        A.tag[p] = DEAD;  // past the live slots of the permuted order
    }

    // ---- deposit (CIC): the core entries reduced across the warp by start
    // cell, the entries of lanes that left their cell added directly
    if constexpr (SHAPE == 1)
        deposit_warp_split<double, 3>(dep, i0, j0, g.nr, wa1, wa2, wb1, wb2, wq * A.m_i2dt, wq * A.idt, wphi, lane,
                                      g.nth, NG, (int)A.ld, A.J0, A.J1, A.J2);

    // ---- histogram of the new keys (warp-aggregated) -----------------------
    if (A.histogram) {
        int hk = (p < n) ? key : -1;
        unsigned peers = __match_any_sync(FULL, hk);
        if (hk >= 0 && lane == __ffs(peers) - 1) atomicAdd(A.count + hk, __popc(peers));
    }
    if (A.cnt9) {
        // old cell = start cell (i0, j0); the key is the new cell; lanes match
        // on cell * 9 + direction (32-bit: see the FP32 push)
        const bool counted = p < n && dep && key >= 0 && key < ncell;
        int dir = 0, c0 = 0;
        if (counted) {
            const int ki = key % g.nr, kj = key / g.nr;
            dir = (kj - j0 + 1) * 3 + (ki - i0 + 1);
            c0 = j0 * g.nr + i0;
        }
        const unsigned mk = counted ? (unsigned)c0 * 9u + (unsigned)dir : 0xffffffffu;
        const unsigned peers = __match_any_sync(FULL, mk);
        if (counted && lane == __ffs(peers) - 1) atomicAdd(A.cnt9 + (int64_t)dir * ncell + c0, (int)__popc(peers));
    }
}

}  // namespace

static Push64Args push64_args(grpic_ctx *ctx, const grpic_particles *in, grpic_particles *p, const int32_t *perm,
                              const int32_t *live, int32_t *cnt9, grpic_fields *f, bool histogram)
{
    Push64Args A;
    A.g = ctx->g;
    A.dt = ctx->prm.dt;
    A.idt = 1.0 / ctx->prm.dt;
    A.m_i2dt = -0.5 / ctx->prm.dt;
    A.n_iter = ctx->prm.n_push_iter;
    for (int k = 0; k < 4; ++k) {
        A.qm[k] = ctx->prm.q_over_m[k];
        A.qw[k] = ctx->prm.q_weight[k];
        A.massive[k] = ctx->prm.massive[k];
    }
    A.n = p->n;
    A.d_count = p->d_count;
    A.r = (double *)p->x1;
    A.th = (double *)p->x2;
    A.u1 = (double *)p->u1;
    A.u2 = (double *)p->u2;
    A.u3 = (double *)p->u3;
    A.tag = p->tag;
    A.perm = perm;
    A.live = live;
    A.count_out = perm ? p->d_count : nullptr;
    A.cnt9 = perm ? cnt9 : nullptr;
    A.in_r = (const double *)in->x1;
    A.in_th = (const double *)in->x2;
    A.in_u1 = (const double *)in->u1;
    A.in_u2 = (const double *)in->u2;
    A.in_u3 = (const double *)in->u3;
    A.in_tag = in->tag;
    A.D0 = (const double *)f->D[0];
    A.D1 = (const double *)f->D[1];
    A.D2 = (const double *)f->D[2];
    A.B0 = (const double *)f->B[0];
    A.B1 = (const double *)f->B[1];
    A.B2 = (const double *)f->B[2];
    A.J0 = (double *)f->J[0];
    A.J1 = (double *)f->J[1];
    A.J2 = (double *)f->J[2];
    A.ld = f->ld;
    A.keys = ctx->d_keys;
    A.count = ctx->d_count;
    A.histogram = histogram ? 1 : 0;
    A.pusher = ctx->prm.pusher;
    A.radiation = ctx->prm.radiation;
    A.gamma_thr = ctx->prm.gamma_thr;
    A.eps_ph = ctx->prm.eps_ph;
    A.pconv = 1.0 - std::exp(-ctx->prm.tau * ctx->prm.dt);
    A.seed = ctx->prm.seed;
    A.step = ctx->step_count;
    A.spawn = ctx->prm.radiation ? ctx->d_spawn : nullptr;
    A.status = ctx->d_status;
    A.tape = nullptr;
    A.tape_ld = 0;
    return A;
}

cudaError_t launch_push64(grpic_ctx *ctx, const grpic_particles *in, grpic_particles *p, const int32_t *perm,
                          const int32_t *live, int32_t *cnt9, grpic_fields *f, bool histogram, cudaStream_t s,
                          int64_t slot0)
{
    Push64Args A = push64_args(ctx, in, p, perm, live, cnt9, f, histogram);
    A.keys = ctx->d_keys + slot0;
    if (p->n <= 0) return cudaSuccess;
    int64_t blocks = (p->n + 255) / 256;
    const bool rad = ctx->prm.radiation != 0;
    if (ctx->prm.shape_order == 3) {
        if (rad)
            push64_kernel<3, true, false><<<(unsigned)blocks, 256, 0, s>>>(A);
        else
            push64_kernel<3, false, false><<<(unsigned)blocks, 256, 0, s>>>(A);
    } else {
        if (rad)
            push64_kernel<1, true, false><<<(unsigned)blocks, 256, 0, s>>>(A);
        else
            push64_kernel<1, false, false><<<(unsigned)blocks, 256, 0, s>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t launch_push64_tape(grpic_ctx *ctx, grpic_particles *p, grpic_fields *f, double *tape, int64_t tape_ld,
                               cudaStream_t s)
{
    if (ctx->prm.shape_order != 1 || ctx->prm.radiation || ctx->prm.pusher != 0 || tape_ld < p->n)
        return cudaErrorInvalidValue;
    Push64Args A = push64_args(ctx, p, p, nullptr, nullptr, nullptr, f, false);
    A.tape = tape;
    A.tape_ld = tape_ld;
    if (p->n <= 0) return cudaSuccess;
    push64_kernel<1, false, true><<<(unsigned)((p->n + 255) / 256), 256, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace grpic
