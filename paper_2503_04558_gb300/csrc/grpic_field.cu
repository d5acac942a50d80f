// grpic_field.cu -- semi-implicit D/B field update (arXiv:2503.04558 Sec. 2.1,
// Eqs. fld-predictor and fld-corrector; discrete forms of App. B).
//
// One kernel launch per stage (the predictor, then n_field_iter correctors).
// A thread owns the six field components of cell (i, j) (their staggered
// locations of Fig. Yee) and evaluates the auxiliary fields E_i, H_i it needs
// from the current iterate (Eqs. auxE, auxH: metric products formed first,
// then the two-point averages), the circulations C_H, C_E (Eqs. D-update,
// B-update) and the new iterate:
//   predictor:  X~ = X^n + dt (C(X^n) - J),  C(X^n) kept for the correctors
//   corrector:  X  = X^n + dt (alpha_s C(X^n) + beta_s C(X~)) - dt J
// The boundary conditions are applied inside the stage: the threads of the
// first and last physical columns also write the guard columns (zero
// derivative copies), D^phi and B^theta are zero on the axis, D^r on the axis
// uses only the interior H_phi edge over the half-width face (Eq. Dr-axis);
// the last stage multiplies by the outer damping factor before the copy.
// J holds the integrated currents J A (the deposit output) and is divided by
// the face areas here.
#include "grpic_internal.cuh"

#include <cuda.h>  // tensor-map types (the encoder is looked up at run time)

namespace grpic {
namespace {

template <typename T>
struct FieldArgs {
    int nr, nth;
    int64_t ld;      // field arrays
    int64_t ldt;     // tables
    size_t slab;
    T dt, as, bs, dth;
    const T *tab;
    const T *col1d;  // dr_prim, dr_dual, damp_int, damp_half
    const T *Xc[6];  // current iterate (read at neighbours)
    const T *Xn[6];  // state at step n (read at the own point)
    T *Cn[6];        // circulations at step n (written by the predictor)
    T *Xo[6];        // output iterate
    const T *J[3];
    int mode;        // 0 predictor, 1 corrector, 2 last corrector (damping)
    int j_lo, j_hi;  // the rows [j_lo, j_hi) the stage updates
};

// the current iterate read from the global arrays A.Xc
template <typename T>
struct GlobalX {
    const FieldArgs<T> &A;
    __device__ __forceinline__ T operator()(int comp, int i, int j) const
    {
        return __ldg(A.Xc[comp] + (size_t)j * A.ld + (i + NG));
    }
};

template <typename T, typename XR = GlobalX<T>>
struct Ctx {
    const FieldArgs<T> &A;
    XR xr;
    __device__ Ctx(const FieldArgs<T> &a) : A(a), xr{a} {}
    __device__ Ctx(const FieldArgs<T> &a, XR r) : A(a), xr(r) {}
    __device__ __forceinline__ T t(int slot, int i, int j) const
    {
        return __ldg(A.tab + slot * A.slab + (size_t)j * A.ldt + (i + NG));
    }
    __device__ __forceinline__ T x(int comp, int i, int j) const { return xr(comp, i, j); }
    // auxiliary fields (App. B); comp order D^r, D^th, D^ph, B^r, B^th, B^ph
    __device__ __forceinline__ T Hr(int i, int j) const
    {
        return t(T_AGRR_BR, i, j) * x(3, i, j) +
               T(0.5) * (t(T_AGRP_BP, i, j) * x(5, i, j) + t(T_AGRP_BP, i - 1, j) * x(5, i - 1, j));
    }
    __device__ __forceinline__ T Hth(int i, int j) const
    {
        return t(T_AGTT_BT, i, j) * x(4, i, j) +
               T(0.5) * (t(T_SGB_DP, i, j) * x(2, i, j) + t(T_SGB_DP, i + 1, j) * x(2, i + 1, j));
    }
    __device__ __forceinline__ T Hph(int i, int j) const
    {
        return t(T_AGPP_BP, i, j) * x(5, i, j) +
               T(0.5) * (t(T_AGRP_BR, i, j) * x(3, i, j) + t(T_AGRP_BR, i + 1, j) * x(3, i + 1, j)) -
               T(0.5) * (t(T_SGB_DT, i, j) * x(1, i, j) + t(T_SGB_DT, i + 1, j) * x(1, i + 1, j));
    }
    __device__ __forceinline__ T Er(int i, int j) const
    {
        return t(T_AGRR_DR, i, j) * x(0, i, j) +
               T(0.5) * (t(T_AGRP_DP, i, j) * x(2, i, j) + t(T_AGRP_DP, i + 1, j) * x(2, i + 1, j));
    }
    __device__ __forceinline__ T Eth(int i, int j) const
    {
        return t(T_AGTT_DT, i, j) * x(1, i, j) -
               T(0.5) * (t(T_SGB_BP, i, j) * x(5, i, j) + t(T_SGB_BP, i - 1, j) * x(5, i - 1, j));
    }
    __device__ __forceinline__ T Eph(int i, int j) const
    {
        return t(T_AGPP_DP, i, j) * x(2, i, j) +
               T(0.5) * (t(T_AGRP_DR, i, j) * x(0, i, j) + t(T_AGRP_DR, i - 1, j) * x(0, i - 1, j)) +
               T(0.5) * (t(T_SGB_BT, i, j) * x(4, i, j) + t(T_SGB_BT, i - 1, j) * x(4, i - 1, j));
    }
};

template <typename T>
__device__ __forceinline__ void store(const FieldArgs<T> &A, int comp, int i, int j, T C, T Jd, bool half_r)
{
    size_t q = (size_t)j * A.ld + (i + NG);
    T v;
    T xn = __ldg(A.Xn[comp] + q);
    if (A.mode == 0) {
        A.Cn[comp][q] = C;
        v = xn + A.dt * (C - Jd);
    } else {
        T cn = __ldg(A.Cn[comp] + q);
        v = xn + A.dt * (A.as * cn + A.bs * C) - Jd * A.dt;
    }
    if (A.mode == 2) v *= __ldg(A.col1d + (half_r ? 3 : 2) * A.ldt + (i + NG));
    T *o = A.Xo[comp] + (size_t)j * A.ld;
    o[i + NG] = v;
    // guard columns: zero-derivative copies of the first / last physical cell
    if (i == 0) {
        o[0] = v;
        o[1] = v;
    }
    int last = half_r ? A.nr - 1 : A.nr;
    if (i == last)
        for (int c = last + 1 + NG; c < A.nr + 2 * NG; ++c) o[c] = v;
}

template <typename T>
__device__ __forceinline__ void store_zero(const FieldArgs<T> &A, int comp, int i, int j, bool half_r)
{
    T *o = A.Xo[comp] + (size_t)j * A.ld;
    o[i + NG] = T(0);
    if (i == 0) {
        o[0] = T(0);
        o[1] = T(0);
    }
    int last = half_r ? A.nr - 1 : A.nr;
    if (i == last)
        for (int c = last + 1 + NG; c < A.nr + 2 * NG; ++c) o[c] = T(0);
}

// the new iterate of the six components of point (i, j) (the stage body):
// the circulations from the current iterate (X), the update of each
// component handed to put.store / put.zero
template <typename T, typename CX, typename PUT>
__device__ __forceinline__ void stage_point(const FieldArgs<T> &A, const CX &X, const PUT &put, int i, int j)
{
    const int nr = A.nr, nth = A.nth;
    size_t qf = (size_t)j * A.ld + (i + NG);
    T drd = __ldg(A.col1d + 1 * A.ldt + (i + NG));
    T drp = __ldg(A.col1d + 0 * A.ldt + (i + NG));

    // D^r at (i+1/2, j): i <= nr-1, all rows (axis rows use one edge)
    if (i <= nr - 1) {
        T hp = (j < nth) ? X.Hph(i, j) : T(0);
        T hm = (j > 0) ? X.Hph(i, j - 1) : T(0);
        T C = (hp - hm) * X.t(T_INV_ADR, i, j);
        T Jd = __ldg(A.J[0] + qf) * X.t(T_INV_ADR, i, j);
        put.store(0, i, j, C, Jd, true);
    }
    if (j < nth) {
        // D^theta at (i, j+1/2)
        T C = (X.Hph(i - 1, j) - X.Hph(i, j)) * X.t(T_INV_ADT, i, j);
        T Jd = __ldg(A.J[1] + qf) * X.t(T_INV_ADT, i, j);
        put.store(1, i, j, C, Jd, false);
        // B^r at (i, j+1/2)
        T Cb = -(X.Eph(i, j + 1) - X.Eph(i, j)) * X.t(T_INV_ABR, i, j);
        put.store(3, i, j, Cb, T(0), false);
    }
    if (j > 0 && j < nth) {
        // D^phi at (i, j)
        T C = ((X.Hth(i, j) - X.Hth(i - 1, j)) * A.dth + (X.Hr(i, j - 1) - X.Hr(i, j)) * drd) * X.t(T_INV_ADP, i, j);
        T Jd = __ldg(A.J[2] + qf) * X.t(T_INV_ADP, i, j);
        put.store(2, i, j, C, Jd, false);
        // B^theta at (i+1/2, j)
        if (i <= nr - 1) {
            T Cb = -(X.Eph(i, j) - X.Eph(i + 1, j)) * X.t(T_INV_ABT, i, j);
            put.store(4, i, j, Cb, T(0), true);
        }
    } else {
        put.zero(2, i, j, false);
        if (i <= nr - 1) put.zero(4, i, j, true);
    }
    // B^phi at (i+1/2, j+1/2)
    if (i <= nr - 1 && j < nth) {
        T C = -((X.Eth(i + 1, j) - X.Eth(i, j)) * A.dth + (X.Er(i, j) - X.Er(i, j + 1)) * drp) * X.t(T_INV_ABP, i, j);
        put.store(5, i, j, C, T(0), true);
    }
}

// the update written to the global arrays A.Xo (and C^n to A.Cn in the predictor)
template <typename T>
struct GlobalPut {
    const FieldArgs<T> &A;
    __device__ __forceinline__ void store(int comp, int i, int j, T C, T Jd, bool half_r) const
    {
        grpic::store(A, comp, i, j, C, Jd, half_r);
    }
    __device__ __forceinline__ void zero(int comp, int i, int j, bool half_r) const
    {
        store_zero(A, comp, i, j, half_r);
    }
};

// latency-bound on its loads: the FP32 stage runs fastest at full occupancy
// (8 CTAs of 256 per SM, 32 registers; 1.85 -> 1.46 ms for the 8 stages at
// 2048^2), the FP64 one is indifferent
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 1) field_stage_kernel(FieldArgs<T> A)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = A.j_lo + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    if (i > A.nr || j >= A.j_hi) return;
    Ctx<T> X(A);
    GlobalPut<T> put{A};
    stage_point(A, X, put, i, j);
}

// ---------------------------------------------------------------------------
// Fused stages (FP32): FZ_NS consecutive stages of the update per launch on a
// tile held in shared memory.  A CTA owns an FZ_OW x FZ_OH rectangle of array
// columns and rows; TMA (cp.async.bulk.tensor) brings the six components of
// the iterate (and, after the first launch, C^n) over the rectangle plus a
// halo of FZ_NS on each side into shared memory.  Stage k of the launch
// updates the points within FZ_NS - 1 - k of the rectangle from the shared
// copy (each stage reads one point beyond the one it writes), so the last
// stage leaves the rectangle exact; it goes to a global buffer.  A stage runs
// in two passes over the tile: the auxiliary fields E_i, H_i into shared
// memory, then the circulations and the update from them.  The table
// slabs are read from global memory (each CTA's slabs stay in L1/L2 over its
// stages); X^n and J at the point itself.  The operations per point are the
// per-stage kernel's (the results agree to FP32 rounding: the compiler
// contracts a few multiply-adds differently in the two kernels).  Two CTAs of
// 512 threads share an SM (110.7 KB of shared memory each), so that one CTA's
// tile load and barriers overlap the other's passes (1.37 -> 1.29 ms per
// update at 2048^2 against one CTA of 1024 threads on 56 x 24 points).
#ifndef GRPIC_FZ_OW
#define GRPIC_FZ_OW 56
#endif
#ifndef GRPIC_FZ_OH
#define GRPIC_FZ_OH 16
#endif
constexpr int FZ_NS = 4, FZ_OW = GRPIC_FZ_OW, FZ_OH = GRPIC_FZ_OH;
constexpr int FZ_BW = FZ_OW + 2 * FZ_NS, FZ_BH = FZ_OH + 2 * FZ_NS;   // 64 x 24 box
constexpr int FZ_BOX = FZ_BW * FZ_BH;
#ifndef GRPIC_FZ_THREADS
#define GRPIC_FZ_THREADS 512
#endif
#ifndef GRPIC_FZ_MINB
#define GRPIC_FZ_MINB 2
#endif
constexpr int FZ_THREADS = GRPIC_FZ_THREADS;
constexpr int FZ_SMEM = (3 * 6 * FZ_BOX) * 4 + 128;   // the iterate, C^n, E and H (floats); the barrier

struct FusedMaps {
    CUtensorMap x[6];   // the iterate at the launch's first stage
    CUtensorMap cn[6];  // C^n (launches after the first)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// the iterate in shared memory: box point (bc, br) holds array column c0 + bc
// and row r0 + br
struct SmemX32 {
    const float *base;
    int c0, r0;
    __device__ __forceinline__ float operator()(int comp, int i, int j) const
    {
        return base[(comp * FZ_BH + (j - r0)) * FZ_BW + (i + NG - c0)];
    }
};

// E_i and H_i of a stage read from the shared tile the stage's first pass
// wrote (components 0..5 = H_r, H_theta, H_phi, E_r, E_theta, E_phi), the
// tables from global memory: the circulation pass of stage_point
struct AuxSmem32 {
    const FieldArgs<float> &A;
    const float *eh;
    int c0, r0;
    __device__ __forceinline__ float a(int k, int i, int j) const
    {
        return eh[(k * FZ_BH + (j - r0)) * FZ_BW + (i + NG - c0)];
    }
    __device__ __forceinline__ float t(int slot, int i, int j) const
    {
        return __ldg(A.tab + slot * A.slab + (size_t)j * A.ldt + (i + NG));
    }
    __device__ __forceinline__ float Hr(int i, int j) const { return a(0, i, j); }
    __device__ __forceinline__ float Hth(int i, int j) const { return a(1, i, j); }
    __device__ __forceinline__ float Hph(int i, int j) const { return a(2, i, j); }
    __device__ __forceinline__ float Er(int i, int j) const { return a(3, i, j); }
    __device__ __forceinline__ float Eth(int i, int j) const { return a(4, i, j); }
    __device__ __forceinline__ float Eph(int i, int j) const { return a(5, i, j); }
};

struct SmemPut32 {
    const FieldArgs<float> &A;
    float *xo;        // the next iterate (box layout)
    float *cn;        // C^n (box layout)
    int c0, r0;
    __device__ __forceinline__ int at(int comp, int col, int j) const
    {
        return (comp * FZ_BH + (j - r0)) * FZ_BW + (col - c0);
    }
    __device__ __forceinline__ void put(int comp, int i, int j, float v, bool half_r) const
    {
        xo[at(comp, i + NG, j)] = v;
        // guard columns: zero-derivative copies of the first / last physical cell
        if (i == 0) {
            if (c0 <= 0) {
                xo[at(comp, 0, j)] = v;
                xo[at(comp, 1, j)] = v;
            }
        }
        const int last = half_r ? A.nr - 1 : A.nr;
        if (i == last)
            for (int c = last + 1 + NG; c < A.nr + 2 * NG; ++c)
                if (c - c0 < FZ_BW) xo[at(comp, c, j)] = v;
    }
    __device__ __forceinline__ void store(int comp, int i, int j, float C, float Jd, bool half_r) const
    {
        const size_t q = (size_t)j * A.ld + (i + NG);
        const int b = at(comp, i + NG, j);
        const float xn = __ldg(A.Xn[comp] + q);
        float v;
        if (A.mode == 0) {
            cn[b] = C;
            v = xn + A.dt * (C - Jd);
        } else {
            v = xn + A.dt * (A.as * cn[b] + A.bs * C) - Jd * A.dt;
        }
        if (A.mode == 2) v *= __ldg(A.col1d + (half_r ? 3 : 2) * A.ldt + (i + NG));
        put(comp, i, j, v, half_r);
    }
    __device__ __forceinline__ void zero(int comp, int i, int j, bool half_r) const { put(comp, i, j, 0.0f, half_r); }
};

// launch of stages [s0, s0 + ns) (ns <= FZ_NS; last_stage = n_field_iter, the
// damped one); A.Xo receives the rectangle's iterate after the last of them,
// A.Cn (global) the rectangle's C^n when s0 == 0
__global__ void __launch_bounds__(FZ_THREADS, GRPIC_FZ_MINB) field_fused32_kernel(FieldArgs<float> A,
                                                                    const __grid_constant__ FusedMaps M, int s0,
                                                                    int ns, int last_stage, int *status)
{
    extern __shared__ __align__(128) unsigned char fz_smem[];
    float *X0 = reinterpret_cast<float *>(fz_smem);
    float *CN = X0 + 6 * FZ_BOX;
    float *EH = CN + 6 * FZ_BOX;
    uint64_t *bar = reinterpret_cast<uint64_t *>(EH + 6 * FZ_BOX);
    const int a0 = blockIdx.x * FZ_OW, row0 = blockIdx.y * FZ_OH;  // the rectangle's first column and row
    const int c0 = a0 - FZ_NS, r0 = row0 - FZ_NS;                   // the box's
    const bool load_cn = s0 > 0;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (load_cn ? 12u : 6u) * FZ_BOX * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                     : "memory");
        for (int k = 0; k < 6; ++k)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                ::"r"(smem_u32(X0 + k * FZ_BOX)), "l"(&M.x[k]), "r"(c0), "r"(r0), "r"(smem_u32(bar))
                : "memory");
        if (load_cn)
            for (int k = 0; k < 6; ++k)
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                    ::"r"(smem_u32(CN + k * FZ_BOX)), "l"(&M.cn[k]), "r"(c0), "r"(r0), "r"(smem_u32(bar))
                    : "memory");
    }
    // wait for the copies (bounded: a copy that never lands latches ETIMEOUT)
    uint32_t done = 0;
    for (int tries = 0; tries < (1 << 22) && !done; ++tries)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(smem_u32(bar))
                     : "memory");
    if (__syncthreads_or(!done)) {  // every thread leaves together
        if (threadIdx.x == 0) atomicCAS(status, 0, (int)GRPIC_ETIMEOUT);
        // a second bounded wait for copies still in flight before the CTA's
        // shared memory is released
        for (int tries = 0; tries < (1 << 22) && !done; ++tries)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done)
                         : "r"(smem_u32(bar))
                         : "memory");
        return;
    }
    // the iterate is updated in place: a stage's first pass reads it (into E
    // and H), its second pass reads only E, H, C^n, X^n and J; the points a
    // stage does not update keep their values.  C^n of the points the
    // predictor does not reach stays 0
    if (!load_cn) {
        for (int e = threadIdx.x; e < 6 * FZ_BOX; e += FZ_THREADS) CN[e] = 0.0f;
        __syncthreads();
    }
    for (int k = 0; k < ns; ++k) {
        const int st = s0 + k;
        FieldArgs<float> B = A;
        B.mode = st == 0 ? 0 : (st == last_stage ? 2 : 1);
        const int w = ns - 1 - k;  // halo this stage still updates
        const Ctx<float, SmemX32> X(B, SmemX32{X0, c0, r0});
        // pass 1: E_i, H_i (Eqs. auxE, auxH) one point beyond the stage's
        // region, each where its own reads stay in the box and the grid: the
        // kinds reading column i + 1 (H_theta, H_phi, E_r) for i in [-1, n_r],
        // those reading column i - 1 (H_r, E_theta, E_phi) for i in [0, n_r + 1]
#pragma unroll
        for (int e = threadIdx.x; e < FZ_BOX; e += FZ_THREADS) {
            const int bc = e % FZ_BW, br = e / FZ_BW;
            const int i = c0 + bc - NG, j = r0 + br;
            if (bc < FZ_NS - w - 1 || bc >= FZ_NS + FZ_OW + w + 1 || br < FZ_NS - w - 1 ||
                br >= FZ_NS + FZ_OH + w + 1 || j < 0 || j > A.nth)
                continue;
            if (bc + 1 < FZ_BW && i >= -1 && i <= A.nr) {
                EH[1 * FZ_BOX + e] = X.Hth(i, j);
                EH[2 * FZ_BOX + e] = X.Hph(i, j);
                EH[3 * FZ_BOX + e] = X.Er(i, j);
            }
            if (bc >= 1 && i >= 0 && i <= A.nr + 1) {
                EH[0 * FZ_BOX + e] = X.Hr(i, j);
                EH[4 * FZ_BOX + e] = X.Eth(i, j);
                EH[5 * FZ_BOX + e] = X.Eph(i, j);
            }
        }
        __syncthreads();
        // pass 2: circulations and the update on the region
        const AuxSmem32 H{B, EH, c0, r0};
        const SmemPut32 put{B, X0, CN, c0, r0};
#pragma unroll
        for (int e = threadIdx.x; e < FZ_BOX; e += FZ_THREADS) {
            const int bc = e % FZ_BW, br = e / FZ_BW;
            const int i = c0 + bc - NG, j = r0 + br;
            if (bc >= FZ_NS - w && bc < FZ_NS + FZ_OW + w && br >= FZ_NS - w && br < FZ_NS + FZ_OH + w && i >= 0 &&
                i <= A.nr && j >= 0 && j <= A.nth)
                stage_point(B, H, put, i, j);
        }
        __syncthreads();
    }
    // the rectangle's iterate (and C^n after the first stage) to global memory
    const float *res = X0;
    for (int e = threadIdx.x; e < FZ_OW * FZ_OH; e += FZ_THREADS) {
        const int col = a0 + e % FZ_OW, j = row0 + e / FZ_OW;
        if (col >= A.ld || j > A.nth) continue;
        const int b = (j - r0) * FZ_BW + (col - c0);
        const size_t q = (size_t)j * A.ld + col;
        for (int comp = 0; comp < 6; ++comp) {
            A.Xo[comp][q] = res[comp * FZ_BOX + b];
            if (!load_cn) A.Cn[comp][q] = CN[comp * FZ_BOX + b];
        }
    }
}

// cuTensorMapEncodeTiled through the runtime's entry-point lookup (the
// library links no driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
    }
    return fn;
}

// a 2D map of one (nth+1) x ld float array with the fused kernel's box
bool encode_field_map(CUtensorMap *m, const float *base, int rows, int64_t ld)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t stride[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {FZ_BW, FZ_BH};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <typename T>
T *fslot(grpic_ctx *ctx, int k, int64_t ld)
{
    size_t n = (size_t)(ctx->g.nth + 1) * ld;
    return (T *)ctx->fscratch + (size_t)k * n;
}

// rows [j_lo, j_hi) of every component are updated (all rows: 0, nth + 1);
// the rows outside are left as they are and feed the range's edge rows
template <typename T>
cudaError_t run_field(grpic_ctx *ctx, grpic_fields *f, const T *tab, const T *col1d, cudaStream_t s, int j_lo,
                      int j_hi)
{
    FieldArgs<T> A;
    A.nr = ctx->g.nr;
    A.nth = ctx->g.nth;
    A.ld = f->ld;
    A.ldt = ctx->g.ld_tab;
    A.slab = ctx->slab;
    A.dt = (T)ctx->prm.dt;
    A.bs = (T)ctx->prm.beta_field;
    A.as = (T)(1.0 - ctx->prm.beta_field);
    A.dth = (T)ctx->g.dth;
    A.tab = tab;
    A.col1d = col1d;
    T *user[6];
    for (int k = 0; k < 3; ++k) {
        user[k] = (T *)f->D[k];
        user[3 + k] = (T *)f->B[k];
        A.J[k] = (const T *)f->J[k];
    }
    T *Cn[6], *buf[2][6];
    for (int k = 0; k < 6; ++k) {
        Cn[k] = fslot<T>(ctx, k, f->ld);
        buf[0][k] = fslot<T>(ctx, 6 + k, f->ld);
        buf[1][k] = fslot<T>(ctx, 12 + k, f->ld);
        A.Xn[k] = user[k];
        A.Cn[k] = Cn[k];
    }
    A.j_lo = j_lo;
    A.j_hi = j_hi;
    dim3 blk(64, 4), grd((A.nr + 1 + 63) / 64, (j_hi - j_lo + 3) / 4);
    int N = ctx->prm.n_field_iter;
    // predictor
    for (int k = 0; k < 6; ++k) {
        A.Xc[k] = user[k];
        A.Xo[k] = buf[0][k];
    }
    A.mode = 0;
    field_stage_kernel<T><<<grd, blk, 0, s>>>(A);
    int cur = 0;
    for (int it = 0; it < N; ++it) {
        bool last = (it == N - 1);
        for (int k = 0; k < 6; ++k) {
            A.Xc[k] = buf[cur][k];
            A.Xo[k] = last ? user[k] : buf[1 - cur][k];
        }
        A.mode = last ? 2 : 1;
        field_stage_kernel<T><<<grd, blk, 0, s>>>(A);
        cur = 1 - cur;
    }
    if (N == 0) {
        // no corrector: damp and copy the predictor result back (a corrector-free
        // step is the forward-Euler predictor alone)
        size_t off = (size_t)j_lo * f->ld, bytes = (size_t)(j_hi - j_lo) * f->ld * sizeof(T);
        for (int k = 0; k < 6; ++k)
            cudaMemcpyAsync(user[k] + off, buf[0][k] + off, bytes, cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

// The FP32 update by fused launches of FZ_NS stages (all rows); false when
// the arrays do not meet the tensor copy's alignment (16-byte base and row
// stride) or the encoder is missing, and the caller takes the per-stage path.
bool run_field_fused32(grpic_ctx *ctx, grpic_fields *f, cudaStream_t s, cudaError_t *err)
{
    const int64_t ld = f->ld;
    const int rows = ctx->g.nth + 1;
    const int N = ctx->prm.n_field_iter;
    if (N < 1 || (ld * (int64_t)sizeof(float)) % 16 != 0 || !encode_fn()) return false;
    float *user[6];
    for (int k = 0; k < 3; ++k) {
        user[k] = (float *)f->D[k];
        user[3 + k] = (float *)f->B[k];
    }
    for (int k = 0; k < 6; ++k)
        if (((uintptr_t)user[k] & 15) != 0) return false;
    if (((uintptr_t)ctx->fscratch & 15) != 0) return false;
    if (cudaFuncSetAttribute(field_fused32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FZ_SMEM) !=
        cudaSuccess)
        return false;
    FieldArgs<float> A;
    A.nr = ctx->g.nr;
    A.nth = ctx->g.nth;
    A.ld = ld;
    A.ldt = ctx->g.ld_tab;
    A.slab = ctx->slab;
    A.dt = (float)ctx->prm.dt;
    A.bs = (float)ctx->prm.beta_field;
    A.as = (float)(1.0 - ctx->prm.beta_field);
    A.dth = (float)ctx->g.dth;
    A.tab = ctx->tab32;
    A.col1d = ctx->col1d32;
    A.mode = 0;
    A.j_lo = 0;
    A.j_hi = rows;
    for (int k = 0; k < 3; ++k) A.J[k] = (const float *)f->J[k];
    float *Cn[6], *buf[2][6];
    for (int k = 0; k < 6; ++k) {
        Cn[k] = fslot<float>(ctx, k, ld);
        buf[0][k] = fslot<float>(ctx, 6 + k, ld);
        buf[1][k] = fslot<float>(ctx, 12 + k, ld);
        A.Xn[k] = user[k];
        A.Cn[k] = Cn[k];
        A.Xc[k] = nullptr;
    }
    FusedMaps M;
    for (int k = 0; k < 6; ++k)
        if (!encode_field_map(&M.cn[k], Cn[k], rows, ld)) return false;
    const dim3 grd((unsigned)((ld + FZ_OW - 1) / FZ_OW), (unsigned)((rows + FZ_OH - 1) / FZ_OH));
    const float *const *src = user;
    int out = 0;
    for (int s0 = 0; s0 <= N; s0 += FZ_NS) {
        for (int k = 0; k < 6; ++k) {
            if (!encode_field_map(&M.x[k], src[k], rows, ld)) return false;
            A.Xo[k] = buf[out][k];
        }
        const int ns = (N + 1 - s0) < FZ_NS ? (N + 1 - s0) : FZ_NS;
        field_fused32_kernel<<<grd, FZ_THREADS, FZ_SMEM, s>>>(A, M, s0, ns, N, ctx->d_status);
        src = buf[out];
        out ^= 1;
    }
    const size_t bytes = (size_t)rows * ld * sizeof(float);
    for (int k = 0; k < 6; ++k) cudaMemcpyAsync(user[k], src[k], bytes, cudaMemcpyDeviceToDevice, s);
    *err = cudaGetLastError();
    return true;
}

}  // namespace

// The FP64 field update from Xn with currents J, every stage's output kept:
// Y[k][0..5] for k = 0 (predictor) .. N (the last corrector, damped) -- the
// iterates the adjoint needs to differentiate the update w.r.t. its tables.
// Xn is not modified; Y buffers are (nth+1) x ld each.
cudaError_t launch_field64_stages(grpic_ctx *ctx, double *const Xn[6], double *const J[3], double *const *Y,
                                  int64_t ld, cudaStream_t s)
{
    FieldArgs<double> A;
    A.nr = ctx->g.nr;
    A.nth = ctx->g.nth;
    A.ld = ld;
    A.ldt = ctx->g.ld_tab;
    A.slab = ctx->slab;
    A.dt = ctx->prm.dt;
    A.bs = ctx->prm.beta_field;
    A.as = 1.0 - ctx->prm.beta_field;
    A.dth = ctx->g.dth;
    A.tab = ctx->tab;
    A.col1d = ctx->col1d;
    for (int k = 0; k < 3; ++k) A.J[k] = J[k];
    for (int k = 0; k < 6; ++k) {
        A.Xn[k] = Xn[k];
        A.Cn[k] = fslot<double>(ctx, k, ld);
    }
    A.j_lo = 0;
    A.j_hi = A.nth + 1;
    dim3 blk(64, 4), grd((A.nr + 1 + 63) / 64, (A.nth + 1 + 3) / 4);
    const int N = ctx->prm.n_field_iter;
    for (int st = 0; st <= N; ++st) {
        for (int k = 0; k < 6; ++k) {
            A.Xc[k] = st == 0 ? Xn[k] : Y[(st - 1) * 6 + k];
            A.Xo[k] = Y[st * 6 + k];
        }
        A.mode = st == 0 ? 0 : (st == N ? 2 : 1);
        field_stage_kernel<double><<<grd, blk, 0, s>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t launch_field64(grpic_ctx *ctx, grpic_fields *f, cudaStream_t s, int j_lo, int j_hi)
{
    if (j_hi < 0) j_hi = ctx->g.nth + 1;
    return run_field<double>(ctx, f, ctx->tab, ctx->col1d, s, j_lo, j_hi);
}

cudaError_t launch_field32(grpic_ctx *ctx, grpic_fields *f, cudaStream_t s, int j_lo, int j_hi)
{
    if (j_hi < 0) j_hi = ctx->g.nth + 1;
    if (ctx->field_fused && j_lo == 0 && j_hi == ctx->g.nth + 1) {
        cudaError_t e = cudaSuccess;
        if (run_field_fused32(ctx, f, s, &e)) return e;
    }
    return run_field<float>(ctx, f, ctx->tab32, ctx->col1d32, s, j_lo, j_hi);
}

}  // namespace grpic
