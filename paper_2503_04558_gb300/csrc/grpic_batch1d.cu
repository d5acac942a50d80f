// grpic_batch1d.cu -- batched 1D spark gaps in one persistent launch.
//
// The pair-production prescription of arXiv:2503.04558 Sec. 4 (Eq.
// optical-depth) on independent radial lines of a monopole magnetosphere.
// One CTA owns one line at a time (taken from a device queue ordered by
// decreasing particle count) and runs every step of the launch for it with
// the line's D^r, A_r and J^r A_r in shared memory, so fields never travel to
// HBM between steps; lines are independent, so no CTA ever waits for another.
// Per step the CTA streams the line's particles in chunks of blockDim: push
// (electric kick along the line, geodesic predictor-corrector in (r, u_r)),
// 1D Esirkepov deposit into shared memory, FP64 emission / conversion
// decisions with Philox4x64-10, then one packed block scan places survivors
// (in order) in the other buffer and the children (in parent order) in a
// staging area that is appended after the survivors at the end of the step.
//
// A line can also be shared by a cluster of two CTAs on two SMs (the largest
// lines otherwise set the time of a step): each pushes one half of the
// line's particles into its own shared J^r A_r, the two halves are summed
// through distributed shared memory in a fixed order so that both CTAs update
// identical copies of D^r, the second CTA's survivors are moved down behind
// the first's and the children follow in parent order: the same line state
// as one CTA would leave, up to the rounding of the current's sum.
#include "grpic_geo.cuh"
#include "grpic_philox.cuh"

#include <cooperative_groups.h>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace grpic {
namespace {

constexpr int MAX_LINES = 4096;

struct B1Args {
    int nl, n;
    double a, r_in, dx1, dt, gthr, eps_ph, Pconv;
    float af, dx1f, dtf;
    float junit, jinv;  // J^r A_r per fixed-point unit of the line current, and its inverse
    // per-particle work kept off the FP64 pipe: r_i in FP32, the FP32 screen of
    // the emission threshold, the conversion probability as a 53-bit integer
    // threshold (bits < ceil(P 2^53) exactly when the uniform is below P)
    const float *rcolf;
    float gthr2s;
    uint64_t pconv53;
    int n_iter;
    float qm[4], qw[4];
    int massive[4];
    uint64_t seed;
    int64_t C, Cs;
    const double *theta, *I0;
    float *D;
    const float *Ar;
    float *JA;
    const double *rcol;  // r at integer positions 0..n
    int32_t *count;
    int32_t *cell[2];
    float *off[2], *ur[2], *up[2];
    uint32_t *tag[2];
    uint64_t *id[2];
    int32_t *s_cell;
    float *s_off, *s_ur, *s_up;
    uint32_t *s_tag;
    uint64_t *s_id;
    const int32_t *order;
    int32_t *queue;
    int cur, nsteps;
    int64_t step0;
    int *status;
    unsigned long long *events;
};

// ---- line geometry in FP64 for the decisions ------------------------------
// gamma^rr, gamma^rphi, gamma^phiphi at (r, theta) (App. A, Eq. gamma-inverse)
__device__ __forceinline__ void ginv64(double a, double r, double s, double c, double &grr, double &grp, double &gpp)
{
    double rho2 = r * r + a * a * c * c;
    double ir = 1.0 / rho2;
    double z = 2.0 * r * ir;
    grr = (a * a + r * r) * ir - z / (1.0 + z);
    grp = a * ir;
    gpp = ir / (s * s);
}

// round(c) as a 64-bit integer for |c| <= 2^32 without a 64-bit conversion
// (those run on the FP64 pipe): c = hi 2^16 + lo with hi = trunc(c / 2^16),
// lo = c - hi 2^16 exact in FP32, then two 32-bit conversions
__device__ __forceinline__ long long fixed_units(float c)
{
    const float hi = truncf(c * (1.0f / 65536.0f));
    const float lo = fmaf(hi, -65536.0f, c);
    return ((long long)__float2int_rz(hi) << 16) + (long long)__float2int_rn(lo);
}

__device__ __forceinline__ float W1f(float d)
{
    d = fabsf(d);
    return d < 1.0f ? 1.0f - d : 0.0f;
}

// block-wide exclusive scan of one int per thread; returns the total.  No
// barrier after the totals are read: successive calls alternate between two
// wsum buffers (a warp can start the call after next only once every thread
// has passed the next call's first barrier, so this call's buffer is free)
__device__ __forceinline__ int block_scan(int v, int *wsum, int &excl)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    excl = wsum[warp] + x - v;
    return wsum[32];
}

struct Kid {
    int32_t cell;
    float off, ur, up;
    uint32_t tag;
    uint64_t id;
};

// CL CTAs per line (1, or 2 as a thread-block cluster)
template <int CL>
__device__ __forceinline__ void b1_body(const B1Args &A)
{
    namespace cg = cooperative_groups;
    extern __shared__ float smem[];
    const int n = A.n;
    // J^r A_r at faces -1..n in fixed point (units of A.junit): integer sums
    // do not depend on the order of the atomics, so a line's current is the
    // same whichever warps and CTAs deposit it
    long long *sJ = reinterpret_cast<long long *>(smem);
    float *sD = reinterpret_cast<float *>(sJ + n + 2);
    float *sA = sD + n;
    int *wsum = (int *)(sA + n);             // two scan buffers of 33 ints (34 apart)
    int *sv = wsum + 68;                     // [0] line, [3] emitted, [4] converted, [5] pushed,
                                             // [6] survivors, [7] children of this CTA
    const int tid = threadIdx.x, B = blockDim.x;
    const int rank = CL > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int64_t CsR = A.Cs / CL;           // staging slots of this CTA

    for (;;) {
        int q;
        if (tid == 0 && rank == 0) sv[0] = atomicAdd(A.queue, 1);
        if constexpr (CL == 1) {
            __syncthreads();
            q = sv[0];
            __syncthreads();
        } else {
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            q = cl.map_shared_rank(sv, 0)[0];
            cl.sync();
        }
        if (q >= A.nl) break;
        const int k = A.order[q];
        const double th = A.theta[k];
        double sd, cd;
        sincos(th, &sd, &cd);
        const float sf = (float)sd, cf = (float)cd;
        const float I0 = (float)A.I0[k];
        for (int i = tid; i < n; i += B) {
            sD[i] = A.D[(size_t)k * n + i];
            sA[i] = A.Ar[(size_t)k * n + i];
        }
        int cnt = A.count[k];
        if (cnt > A.C) cnt = (int)A.C;
        if (cnt < 0) cnt = 0;
        const size_t base = (size_t)k * A.C, sbase = (size_t)k * A.Cs;
        for (int st = 0; st < A.nsteps; ++st) {
            const int64_t step = A.step0 + st;
            const int src = (A.cur + st) & 1, dst = src ^ 1;
            for (int i = tid; i < n + 2; i += B) sJ[i] = 0;
            if (tid == 0) {
                sv[3] = 0;
                sv[4] = 0;
                sv[5] = cnt;
            }
            __syncthreads();
            // this CTA's part of the line: whole chunks of B particles, the first
            // half of the chunks to rank 0; its survivors go to [lo, ...) for now
            const int nch = (cnt + B - 1) / B, per = (nch + CL - 1) / CL;
            const int lo = min(cnt, rank * per * B), hi = min(cnt, (rank + 1) * per * B);
            // running write offsets of the survivors and of the children: every
            // thread advances its own copy by the block totals of each chunk
            int wp = 0, sp0 = 0;
            for (int cb = lo; cb < hi; cb += B) {
                const int idx = cb + tid;
                bool alive = false;
                int napp = 0;
                Kid kid[2];
                int32_t ci = 0;
                float o = 0.f, ur = 0.f, up = 0.f;
                uint32_t tg = DEAD;
                uint64_t pid = 0;
                if (idx < hi) {
                    size_t p = base + idx;
                    ci = A.cell[src][p];
                    o = A.off[src][p];
                    ur = A.ur[src][p];
                    up = A.up[src][p];
                    tg = A.tag[src][p];
                    pid = A.id[src][p];
                }
                if (idx < hi && !(tg & DEAD) && ci >= 0 && ci < n) {
                    const int sp = tg & 3u;
                    const bool massive = A.massive[sp] != 0, charged = A.qm[sp] != 0.0f;
                    const float rcf = A.rcolf[ci];
                    const float d0 = rcf * expm1f(o * A.dx1f);  // r - r_i
                    if (massive && charged) {
                        // electric part of the Boris step along the line
                        float xi = o - 0.5f, f = xi;
                        int is = ci;
                        if (xi < 0.0f) {
                            is = ci - 1;
                            f = xi + 1.0f;
                        }
                        int a0 = min(max(is, 0), n - 1), a1 = min(max(is + 1, 0), n - 1);
                        float Dp = (1.0f - f) * sD[a0] + f * sD[a1];
                        float r = rcf + d0;
                        float rho2 = r * r + A.af * A.af * cf * cf;
                        float opz = 1.0f + 2.0f * r / rho2;
                        ur += A.qm[sp] * rsqrtf(opz) * A.dtf * opz * Dp;
                    }
                    const float eps = massive ? 1.0f : 0.0f;
                    KSGeo<float> m;
                    RhsT<float> f0, ft;
                    ks_geo_sc<float>(A.af, rcf + d0, sf, cf, m);
                    geo_rhs_m<float, float>(m, eps, ur, 0.0f, up, f0);
                    float dl = d0 + A.dtf * f0.xr, u1 = ur + A.dtf * f0.ur;
                    const float h = 0.5f * A.dtf;
                    for (int it = 0; it < A.n_iter; ++it) {
                        ks_geo_sc<float>(A.af, rcf + dl, sf, cf, m);
                        geo_rhs_m<float, float>(m, eps, u1, 0.0f, up, ft);
                        dl = d0 + h * (ft.xr + f0.xr);
                        u1 = ur + h * (ft.ur + f0.ur);
                    }
                    float on = log1pf(dl / rcf) / A.dx1f;
                    if (!(isfinite(on) && isfinite(u1) && rcf + dl > 0.0f)) {
                        set_status(A.status, GRPIC_ENAN);
                    } else {
                        int di = (int)floorf(on);
                        if (di < -1 || di > 1) {
                            set_status(A.status, GRPIC_ERANGE);
                        } else {
                            if (A.qw[sp] != 0.0f) {
                                // 1D Esirkepov: J A(face f) -= (q/dt) sum_{k'<=f} (S1 - S0)
                                float acc = 0.0f, cq = -A.qw[sp] / A.dtf;
#pragma unroll
                                for (int w = 0; w < 4; ++w) {
                                    acc += W1f(on - (float)(w - 1)) - W1f(o - (float)(w - 1));
                                    int face = ci - 1 + w;
                                    if (acc != 0.0f && face >= -1 && face <= n)
                                        atomicAdd(reinterpret_cast<unsigned long long *>(&sJ[face + 1]),
                                                  (unsigned long long)fixed_units(cq * acc * A.jinv));
                                }
                            }
                            int ni = ci + di;
                            float no = on - (float)di;
                            if (no >= 1.0f) no = 0x1.fffffep-1f;
                            if (no < 0.0f) no = 0.0f;
                            ur = u1;
                            if (ni >= 0 && ni < n) {
                                alive = true;
                                ci = ni;
                                o = no;
                                // FP64 decisions at the new position
                                if (massive && charged) {
                                    // FP32 screen, FP64 decision inside the ambiguity band
                                    float rf = A.rcolf[ci] * (1.0f + expm1f(o * A.dx1f));
                                    float rho2 = rf * rf + A.af * A.af * cf * cf, ir = 1.0f / rho2, z = 2.0f * rf * ir;
                                    float gr = (A.af * A.af + rf * rf) * ir - z / (1.0f + z), gp = A.af * ir,
                                          gq = ir / (sf * sf);
                                    float G2 = 1.0f + gr * ur * ur + 2.0f * gp * ur * up + gq * up * up;
                                    if (G2 >= A.gthr2s) {
                                        double rd = A.rcol[ci] * exp((double)o * A.dx1), grr, grp, gpp;
                                        ginv64(A.a, rd, sd, cd, grr, grp, gpp);
                                        double urd = ur, upd = up;
                                        double G = sqrt(1.0 + grr * urd * urd + 2.0 * grp * urd * upd + gpp * upd * upd);
                                        if (G >= A.gthr) {
                                            double pm = sqrt(G * G - 1.0), Gn = G - A.eps_ph;
                                            double pm2 = sqrt(Gn * Gn - 1.0), sc = pm2 / pm;
                                            kid[0].cell = ci;
                                            kid[0].off = o;
                                            kid[0].ur = (float)(A.eps_ph * urd / pm);
                                            kid[0].up = (float)(A.eps_ph * upd / pm);
                                            kid[0].tag = 3u;
                                            kid[0].id = child_id(pid, step, 0);
                                            ur = (float)(urd * sc);
                                            up = (float)(upd * sc);
                                            napp = 1;
                                        }
                                    }
                                } else if (!massive) {
                                    // the draw first: it fails for all but ~tau dt of the
                                    // photons, which then skip the FP64 energy (the same
                                    // decision: both conditions must hold)
                                    const bool hit = uniform53_bits(A.seed, pid, step, 1) < A.pconv53;
                                    double e = 0.0, urd = ur, upd = up;
                                    if (hit) {
                                        double rd = A.rcol[ci] * exp((double)o * A.dx1), grr, grp, gpp;
                                        ginv64(A.a, rd, sd, cd, grr, grp, gpp);
                                        e = sqrt(grr * urd * urd + 2.0 * grp * urd * upd + gpp * upd * upd);
                                    }
                                    if (e > 2.0 && hit) {
                                        double s = sqrt(0.25 * e * e - 1.0) / e;
                                        for (int w = 0; w < 2; ++w) {
                                            kid[w].cell = ci;
                                            kid[w].off = o;
                                            kid[w].ur = (float)(s * urd);
                                            kid[w].up = (float)(s * upd);
                                            kid[w].tag = (uint32_t)w;
                                            kid[w].id = child_id(pid, step, 1 + w);
                                        }
                                        napp = 2;
                                        alive = false;
                                    }
                                }
                            }
                        }
                    }
                }
                // placement: survivors in order, children in parent order
                int excl;
                int tot = block_scan((alive ? 1 : 0) | (napp << 16), wsum + (((cb - lo) / B) & 1) * 34, excl);
                if (alive) {
                    size_t d = base + lo + wp + (excl & 0xffff);
                    A.cell[dst][d] = ci;
                    A.off[dst][d] = o;
                    A.ur[dst][d] = ur;
                    A.up[dst][d] = up;
                    A.tag[dst][d] = tg;
                    A.id[dst][d] = pid;
                }
                int ap = sp0 + (excl >> 16);
                for (int w = 0; w < napp; ++w) {
                    if (ap + w < CsR) {
                        size_t d = sbase + rank * CsR + ap + w;
                        A.s_cell[d] = kid[w].cell;
                        A.s_off[d] = kid[w].off;
                        A.s_ur[d] = kid[w].ur;
                        A.s_up[d] = kid[w].up;
                        A.s_tag[d] = kid[w].tag;
                        A.s_id[d] = kid[w].id;
                    }
                }
                if (napp == 1) atomicAdd(&sv[3], 1);
                if (napp == 2) atomicAdd(&sv[4], 1);
                wp += tot & 0xffff;
                sp0 += tot >> 16;
            }
            __syncthreads();  // the staging writes, the J atomics and the counters are complete
            if constexpr (CL == 1) {
                // children after the survivors
                const int wptr = wp, sptr = sp0;
                int nap = min(sptr, (int)A.Cs);
                int room = (int)(A.C - wptr);
                int ncopy = min(nap, room);
                if (tid == 0 && ncopy < sptr) set_status(A.status, GRPIC_EOVERFLOW);
                for (int j = tid; j < ncopy; j += B) {
                    size_t s = sbase + j, d = base + wptr + j;
                    A.cell[dst][d] = A.s_cell[s];
                    A.off[dst][d] = A.s_off[s];
                    A.ur[dst][d] = A.s_ur[s];
                    A.up[dst][d] = A.s_up[s];
                    A.tag[dst][d] = A.s_tag[s];
                    A.id[dst][d] = A.s_id[s];
                }
                cnt = wptr + ncopy;
                // field: d(A D)/dt = I0 - J A
                for (int i = tid; i < n; i += B) sD[i] += A.dtf * (I0 - __ll2float_rn(sJ[i + 1]) * A.junit) / sA[i];
                if (A.JA && st == A.nsteps - 1)
                    for (int i = tid; i < n + 2; i += B) A.JA[(size_t)k * (n + 2) + i] = __ll2float_rn(sJ[i]) * A.junit;
            } else {
                cg::cluster_group cl = cg::this_cluster();
                if (tid == 0) {
                    sv[6] = wp;
                    sv[7] = sp0;
                }
                cl.sync();  // both halves pushed: J, counts and staging complete
                const int *v0 = cl.map_shared_rank(sv, 0), *v1 = cl.map_shared_rank(sv, 1);
                const int S0 = v0[6], S1 = v1[6];
                const int K0 = (int)min((int64_t)v0[7], CsR), K1 = (int)min((int64_t)v1[7], CsR);
                // field with the current of the whole line, summed in rank order so
                // that both copies of D^r stay identical
                const long long *J0 = cl.map_shared_rank(sJ, 0), *J1 = cl.map_shared_rank(sJ, 1);
                for (int i = tid; i < n; i += B)
                    sD[i] += A.dtf * (I0 - __ll2float_rn(J0[i + 1] + J1[i + 1]) * A.junit) / sA[i];
                if (A.JA && st == A.nsteps - 1 && rank == 0)
                    for (int i = tid; i < n + 2; i += B)
                        A.JA[(size_t)k * (n + 2) + i] = __ll2float_rn(J0[i] + J1[i]) * A.junit;
                // rank 1's survivors (written from its first particle's slot) move
                // down behind rank 0's, a chunk at a time: every chunk is read
                // before it is written and its destination lies below the next
                // chunk's source, so the move is safe in increasing order
                if (rank == 1 && S0 < lo) {
                    for (int c0 = 0; c0 < S1; c0 += B) {
                        const int q2 = c0 + tid;
                        const bool v = q2 < S1;
                        int32_t mc = 0;
                        float mo = 0.f, mu = 0.f, mp = 0.f;
                        uint32_t mt = 0;
                        uint64_t mi = 0;
                        if (v) {
                            const size_t s2 = base + lo + q2;
                            mc = A.cell[dst][s2];
                            mo = A.off[dst][s2];
                            mu = A.ur[dst][s2];
                            mp = A.up[dst][s2];
                            mt = A.tag[dst][s2];
                            mi = A.id[dst][s2];
                        }
                        __syncthreads();
                        if (v) {
                            const size_t d2 = base + S0 + q2;
                            A.cell[dst][d2] = mc;
                            A.off[dst][d2] = mo;
                            A.ur[dst][d2] = mu;
                            A.up[dst][d2] = mp;
                            A.tag[dst][d2] = mt;
                            A.id[dst][d2] = mi;
                        }
                        __syncthreads();
                    }
                }
                cl.sync();  // survivors in place, the remote J and counts read
                // children after all survivors: rank 0's, then rank 1's
                const int Stot = S0 + S1, room = (int)(A.C - Stot);
                const int c0n = min(K0, max(room, 0)), c1n = min(K1, max(room - c0n, 0));
                if (tid == 0 && rank == 0 && c0n + c1n < v0[7] + v1[7]) set_status(A.status, GRPIC_EOVERFLOW);
                const int mine = rank == 0 ? c0n : c1n, at = Stot + (rank == 0 ? 0 : c0n);
                for (int j = tid; j < mine; j += B) {
                    size_t s2 = sbase + rank * CsR + j, d2 = base + at + j;
                    A.cell[dst][d2] = A.s_cell[s2];
                    A.off[dst][d2] = A.s_off[s2];
                    A.ur[dst][d2] = A.s_ur[s2];
                    A.up[dst][d2] = A.s_up[s2];
                    A.tag[dst][d2] = A.s_tag[s2];
                    A.id[dst][d2] = A.s_id[s2];
                }
                cnt = Stot + c0n + c1n;
            }
            if (tid == 0) {
                if (sv[3]) atomicAdd(&A.events[0], (unsigned long long)sv[3]);
                if (sv[4]) atomicAdd(&A.events[1], (unsigned long long)sv[4]);
                if (rank == 0) atomicAdd(&A.events[2], (unsigned long long)sv[5]);  // particles pushed this step
            }
            if constexpr (CL == 1)
                __syncthreads();
            else
                cg::this_cluster().sync();  // the line's next state complete before the next step reads it
        }
        if (rank == 0) {
            for (int i = tid; i < n; i += B) A.D[(size_t)k * n + i] = sD[i];
            if (tid == 0) A.count[k] = cnt;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) b1_kernel(B1Args A) { b1_body<1>(A); }
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(1024) b1_kernel_cl2(B1Args A) { b1_body<2>(A); }

// order the lines by decreasing particle count (ties by index) and reset the
// work queue: one block, bitonic network in shared memory
__global__ void order_kernel(const int32_t *count, int nl, int32_t *order, int32_t *queue)
{
    __shared__ unsigned long long key[MAX_LINES];
    int N = 1;
    while (N < nl) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        key[i] = i < nl ? ((unsigned long long)(0x7fffffffu - (uint32_t)count[i]) << 32) | (uint32_t)i : ~0ULL;
    __syncthreads();
    for (int kk = 2; kk <= N; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & kk) == 0;
                    unsigned long long a = key[i], b = key[l];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < nl; i += blockDim.x) order[i] = (int32_t)(key[i] & 0xffffffffu);
    if (threadIdx.x == 0) *queue = 0;
}

// A_r = sqrt(gamma) at (r_{i+1/2}, theta_k) and the monopole D^r there (App. C)
__global__ void b1_fields_kernel(int nl, int n, double a, double r_in, double dx1, double B0, const double *theta,
                                 float *Ar, float *D)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (i >= n || k >= nl) return;
    double r = r_in * exp((i + 0.5) * dx1), th = theta[k];
    double s, c;
    sincos(th, &s, &c);
    KS m;
    ks_point(a, r, th, m);
    double rho2 = r * r + a * a * c * c, rho4 = rho2 * rho2;
    double Er = -B0 * 2.0 * a * r * c / rho4;
    double sgBth = -B0 * 2.0 * a * a * r * s * s * c / rho4;  // sqrt(gamma) B^theta
    double Eph = -m.beta * sgBth;                             // E_phi - e_{phi r theta} beta B^theta
    Ar[(size_t)k * n + i] = (float)m.sqrtg;
    D[(size_t)k * n + i] = (float)((m.gi_rr * Er + m.gi_rp * Eph) / m.alpha);
}

}  // namespace
}  // namespace grpic

struct grpic_batch1d_ctx {
    grpic_batch1d_params p;
    double *rcol;
    float *rcolf;
    float *Ar;
    int32_t *order, *queue;
    int *status;
    int32_t *s_cell;
    float *s_off, *s_ur, *s_up;
    uint32_t *s_tag;
    uint64_t *s_id;
    int64_t Cs;
    int block, per_sm, cluster, sms;  // launch shape: threads per CTA, CTAs per SM, CTAs per line
    size_t smem;
    // CUDA graph of one run (line order + persistent kernel) and what it was built for
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    cudaGraphNode_t g_b1;
    const void *gkey[20];
    int gshape[3];
};

using namespace grpic;

namespace {

B1Args make_args(grpic_batch1d_ctx *c, grpic_lines *L, int nsteps, int64_t step0)
{
    B1Args A;
    memset(&A, 0, sizeof A);
    const grpic_batch1d_params &p = c->p;
    A.nl = p.n_lines;
    A.n = p.n_cells;
    A.a = p.a;
    A.af = (float)p.a;
    A.r_in = p.r_in;
    A.dx1 = std::log(p.r_out / p.r_in) / p.n_cells;
    A.dx1f = (float)A.dx1;
    A.dt = p.dt;
    A.dtf = (float)p.dt;
    A.n_iter = p.n_push_iter;
    for (int s = 0; s < 4; ++s) {
        A.qm[s] = (float)p.q_over_m[s];
        A.qw[s] = (float)p.q_weight[s];
        A.massive[s] = p.massive[s];
    }
    A.gthr = p.gamma_thr;
    A.eps_ph = p.eps_ph;
    A.Pconv = -std::expm1(-p.tau * p.dt);
    A.seed = p.seed;
    A.C = p.capacity;
    A.Cs = c->Cs;
    // fixed-point unit of the current: 2^-32 of the largest contribution of
    // one particle (|q w| / dt), so that 2^30 particles cannot overflow a sum
    double qmax = 0.0;
    for (int s = 0; s < 4; ++s) qmax = std::max(qmax, std::fabs(p.q_weight[s]));
    const double unit = qmax > 0.0 ? qmax / p.dt * std::ldexp(1.0, -32) : 1.0;
    A.junit = (float)unit;
    A.jinv = (float)(1.0 / unit);
    A.rcolf = c->rcolf;
    A.gthr2s = (float)(p.gamma_thr * p.gamma_thr) * 0.9999f;
    A.pconv53 = (uint64_t)std::ceil(A.Pconv * 9007199254740992.0);
    A.theta = L->theta;
    A.I0 = L->I0;
    A.D = L->D;
    A.Ar = c->Ar;
    A.JA = L->JA;
    A.rcol = c->rcol;
    A.count = L->count;
    for (int b = 0; b < 2; ++b) {
        A.cell[b] = L->cell[b];
        A.off[b] = L->off[b];
        A.ur[b] = L->ur[b];
        A.up[b] = L->up[b];
        A.tag[b] = L->tag[b];
        A.id[b] = L->id[b];
    }
    A.s_cell = c->s_cell;
    A.s_off = c->s_off;
    A.s_ur = c->s_ur;
    A.s_up = c->s_up;
    A.s_tag = c->s_tag;
    A.s_id = c->s_id;
    A.order = c->order;
    A.queue = c->queue;
    A.cur = L->cur;
    A.nsteps = nsteps;
    A.step0 = step0;
    A.status = c->status;
    A.events = L->events;
    return A;
}

bool lines_ok(const grpic_lines *L)
{
    if (!L || !L->theta || !L->I0 || !L->D || !L->count || !L->events || (L->cur != 0 && L->cur != 1)) return false;
    for (int b = 0; b < 2; ++b)
        if (!L->cell[b] || !L->off[b] || !L->ur[b] || !L->up[b] || !L->tag[b] || !L->id[b]) return false;
    return true;
}

// CTAs of a launch: per_sm on every SM; with two CTAs per line, as many
// clusters as can be resident at once (a cluster needs two SMs of one GPC)
int b1_grid(grpic_batch1d_ctx *c, int block, int per_sm, int cluster)
{
    if (cluster == 1) return c->sms * per_sm;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)(c->sms * per_sm));
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = c->smem;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (void *)b1_kernel_cl2, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return 2 * std::min(ncl, c->sms * per_sm / 2);
}

const void *b1_func(int cluster) { return cluster == 2 ? (const void *)b1_kernel_cl2 : (const void *)b1_kernel; }

bool shape_ok(grpic_batch1d_ctx *c, int block, int per_sm, int cluster)
{
    if (block < 32 || block > 1024 || block % 32 != 0 || per_sm < 1 || (cluster != 1 && cluster != 2)) return false;
    int maxb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, b1_kernel, block, c->smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return per_sm <= maxb && b1_grid(c, block, per_sm, cluster) >= cluster;
}

cudaError_t launch_b1(grpic_batch1d_ctx *c, grpic_lines *L, int nsteps, int64_t step0, int block, int per_sm,
                      int cluster, cudaStream_t s)
{
    order_kernel<<<1, 1024, 0, s>>>(L->count, c->p.n_lines, c->order, c->queue);
    B1Args A = make_args(c, L, nsteps, step0);
    const int grid = b1_grid(c, block, per_sm, cluster);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (cluster == 2)
        b1_kernel_cl2<<<grid, block, c->smem, s>>>(A);
    else
        b1_kernel<<<grid, block, c->smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

grpic_status grpic_batch1d_init(const grpic_batch1d_params *p, grpic_batch1d_ctx **out)
{
    if (!out) return GRPIC_EINVAL;
    *out = nullptr;
    if (!p || p->n_lines < 1 || p->n_lines > MAX_LINES || p->n_cells < 4 || p->n_cells > 8192 ||
        !(p->a >= 0.0 && p->a < 1.0) || !(p->r_in > 0.0 && p->r_out > p->r_in) || !(p->dt > 0.0) ||
        p->n_push_iter < 0 || p->n_push_iter > 64 || p->capacity < 1 || p->capacity > (int64_t)1 << 30 ||
        !(p->gamma_thr > 1.0) || !(p->eps_ph > 0.0) || !(p->tau >= 0.0) || p->gamma_thr <= p->eps_ph + 1.0)
        return GRPIC_EINVAL;
    grpic_batch1d_ctx *c = new (std::nothrow) grpic_batch1d_ctx();
    if (!c) return GRPIC_ENOMEM;
    memset((void *)c, 0, sizeof *c);
    c->p = *p;
    int n = p->n_cells;
    c->Cs = p->capacity / 2 > 0 ? p->capacity / 2 : 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    c->smem = sizeof(long long) * ((size_t)n + 2) + sizeof(float) * 2 * (size_t)n + sizeof(int) * 80;
    size_t ns = (size_t)p->n_lines * c->Cs;
    cudaError_t e = cudaMalloc(&c->rcol, sizeof(double) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&c->rcolf, sizeof(float) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&c->Ar, sizeof(float) * (size_t)p->n_lines * n);
    if (e == cudaSuccess) e = cudaMalloc(&c->order, sizeof(int32_t) * p->n_lines);
    if (e == cudaSuccess) e = cudaMalloc(&c->queue, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->s_cell, sizeof(int32_t) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&c->s_off, sizeof(float) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&c->s_ur, sizeof(float) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&c->s_up, sizeof(float) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&c->s_tag, sizeof(uint32_t) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&c->s_id, sizeof(uint64_t) * ns);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(b1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(b1_kernel_cl2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem);
    if (e != cudaSuccess) {
        grpic_batch1d_destroy(c);
        return GRPIC_ENOMEM;
    }
    std::vector<double> r(n + 1);
    double dx1 = std::log(p->r_out / p->r_in) / n;
    for (int i = 0; i <= n; ++i) r[i] = p->r_in * std::exp(i * dx1);
    cudaMemcpy(c->rcol, r.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice);
    std::vector<float> rf(r.begin(), r.end());
    cudaMemcpy(c->rcolf, rf.data(), sizeof(float) * (n + 1), cudaMemcpyHostToDevice);
    cudaMemset(c->status, 0, sizeof(int) * 4);
    // default launch shape until the tuner picks one
    c->block = 256;
    c->per_sm = 2;
    c->cluster = 1;
    int maxb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, b1_kernel, c->block, c->smem);
    if (maxb < 1) {
        grpic_batch1d_destroy(c);
        return GRPIC_EINVAL;
    }
    if (c->per_sm > maxb) c->per_sm = maxb;
    *out = c;
    return GRPIC_OK;
}

grpic_status grpic_batch1d_init_fields(grpic_batch1d_ctx *c, grpic_lines *L, void *stream)
{
    if (!c || !lines_ok(L)) return GRPIC_EINVAL;
    const grpic_batch1d_params &p = c->p;
    dim3 blk(256), grd((p.n_cells + 255) / 256, p.n_lines);
    b1_fields_kernel<<<grd, blk, 0, (cudaStream_t)stream>>>(p.n_lines, p.n_cells, p.a, p.r_in,
                                                             std::log(p.r_out / p.r_in) / p.n_cells, p.B0, L->theta,
                                                             c->Ar, L->D);
    return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}

grpic_status grpic_batch1d_run(grpic_batch1d_ctx *c, grpic_lines *L, int nsteps, int64_t step0, void *stream)
{
    if (!c || !lines_ok(L) || nsteps < 0) return GRPIC_EINVAL;
    if (nsteps == 0) return GRPIC_OK;
    cudaError_t e = launch_b1(c, L, nsteps, step0, c->block, c->per_sm, c->cluster, (cudaStream_t)stream);
    if (e != cudaSuccess) return GRPIC_ECUDA;
    if (nsteps & 1) L->cur ^= 1;
    return GRPIC_OK;
}

grpic_status grpic_batch1d_tune(grpic_batch1d_ctx *c, grpic_lines *L, int trial_steps, int64_t step0,
                                int64_t *steps_done, int32_t best[3], void *stream)
{
    if (!c || !lines_ok(L) || trial_steps < 1 || !steps_done || !best) return GRPIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks[4] = {128, 256, 512, 1024};
    const int persm[3] = {1, 2, 4};
    float best_ms = 1e30f;
    int bb = c->block, bp = c->per_sm, bc = c->cluster;
    int64_t done = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int cl = 1; cl <= 2; ++cl) {
      for (int b : blocks) {
        for (int ps : persm) {
            if (!shape_ok(c, b, ps, cl)) continue;
            cudaEventRecord(e0, s);
            if (launch_b1(c, L, trial_steps, step0 + done, b, ps, cl, s) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return GRPIC_ECUDA;
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            if (trial_steps & 1) L->cur ^= 1;
            done += trial_steps;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                bb = b;
                bp = ps;
                bc = cl;
            }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->block = bb;
    c->per_sm = bp;
    c->cluster = bc;
    best[0] = bb;
    best[1] = bp;
    best[2] = bc;
    *steps_done = done;
    return GRPIC_OK;
}

grpic_status grpic_batch1d_set_launch(grpic_batch1d_ctx *c, int32_t threads, int32_t ctas_per_sm, int32_t ctas_per_line)
{
    if (!c || !shape_ok(c, threads, ctas_per_sm, ctas_per_line)) return GRPIC_EINVAL;
    c->block = threads;
    c->per_sm = ctas_per_sm;
    c->cluster = ctas_per_line;
    return GRPIC_OK;
}

grpic_status grpic_batch1d_run_graph(grpic_batch1d_ctx *c, grpic_lines *L, int nsteps, int64_t step0, void *stream)
{
    if (!c || !lines_ok(L) || nsteps < 0) return GRPIC_EINVAL;
    if (nsteps == 0) return GRPIC_OK;
    const void *key[20] = {L->theta, L->I0, L->D, L->JA, L->count, L->events, L->cell[0], L->cell[1], L->off[0],
                           L->off[1], L->ur[0], L->ur[1], L->up[0], L->up[1], L->tag[0], L->tag[1], L->id[0],
                           L->id[1], nullptr, nullptr};
    B1Args A = make_args(c, L, nsteps, step0);
    cudaKernelNodeParams pb;
    memset(&pb, 0, sizeof pb);
    void *bargs[] = {&A};
    pb.func = (void *)b1_func(c->cluster);
    pb.gridDim = dim3((unsigned)b1_grid(c, c->block, c->per_sm, c->cluster));
    pb.blockDim = dim3((unsigned)c->block);
    pb.sharedMemBytes = (unsigned)c->smem;
    pb.kernelParams = bargs;
    cudaError_t e = cudaSuccess;
    if (pb.gridDim.x < 1) return GRPIC_ECUDA;
    bool same = c->gexec && memcmp(key, c->gkey, sizeof key) == 0 && c->gshape[0] == c->block &&
                c->gshape[1] == c->per_sm && c->gshape[2] == c->cluster;
    if (same) {
        // only the run's arguments (steps, first step, current buffer) change
        e = cudaGraphExecKernelNodeSetParams(c->gexec, c->g_b1, &pb);
    } else {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->gexec = nullptr;
        c->graph = nullptr;
        e = cudaGraphCreate(&c->graph, 0);
        cudaGraphNode_t n_order = nullptr;
        int32_t *cnt = L->count, *ord = c->order, *que = c->queue;
        int nl = c->p.n_lines;
        void *oargs[] = {&cnt, &nl, &ord, &que};
        cudaKernelNodeParams po;
        memset(&po, 0, sizeof po);
        po.func = (void *)order_kernel;
        po.gridDim = dim3(1);
        po.blockDim = dim3(1024);
        po.kernelParams = oargs;
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n_order, c->graph, nullptr, 0, &po);
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&c->g_b1, c->graph, &n_order, 1, &pb);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, c->graph, 0);
        if (e != cudaSuccess) {
            if (c->graph) cudaGraphDestroy(c->graph);
            c->graph = nullptr;
            c->gexec = nullptr;
            return GRPIC_ECUDA;
        }
        memcpy(c->gkey, key, sizeof key);
        c->gshape[0] = c->block;
        c->gshape[1] = c->per_sm;
        c->gshape[2] = c->cluster;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(c->gexec, (cudaStream_t)stream);
    if (e != cudaSuccess) return GRPIC_ECUDA;
    if (nsteps & 1) L->cur ^= 1;
    return GRPIC_OK;
}

grpic_status grpic_batch1d_sync(grpic_batch1d_ctx *c, void *stream)
{
    if (!c) return GRPIC_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GRPIC_ECUDA;
    int st = 0;
    if (cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GRPIC_ECUDA;
    if (st) cudaMemset(c->status, 0, sizeof(int));
    return (grpic_status)st;
}

void grpic_batch1d_destroy(grpic_batch1d_ctx *c)
{
    if (!c) return;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    void *ptrs[] = {c->rcol, c->rcolf, c->Ar, c->order, c->queue, c->status, c->s_cell,
                    c->s_off, c->s_ur, c->s_up, c->s_tag, c->s_id};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete c;
}

}  // extern "C"
