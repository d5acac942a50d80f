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

template <typename T>
struct Ctx {
    const FieldArgs<T> &A;
    __device__ Ctx(const FieldArgs<T> &a) : A(a) {}
    __device__ __forceinline__ T t(int slot, int i, int j) const
    {
        return __ldg(A.tab + slot * A.slab + (size_t)j * A.ldt + (i + NG));
    }
    __device__ __forceinline__ T x(int comp, int i, int j) const
    {
        return __ldg(A.Xc[comp] + (size_t)j * A.ld + (i + NG));
    }
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
    const int nr = A.nr, nth = A.nth;
    size_t qt = (size_t)j * A.ldt + (i + NG);
    size_t qf = (size_t)j * A.ld + (i + NG);
    T drd = __ldg(A.col1d + 1 * A.ldt + (i + NG));
    T drp = __ldg(A.col1d + 0 * A.ldt + (i + NG));

    // D^r at (i+1/2, j): i <= nr-1, all rows (axis rows use one edge)
    if (i <= nr - 1) {
        T hp = (j < nth) ? X.Hph(i, j) : T(0);
        T hm = (j > 0) ? X.Hph(i, j - 1) : T(0);
        T C = (hp - hm) * X.t(T_INV_ADR, i, j);
        T Jd = __ldg(A.J[0] + qf) * X.t(T_INV_ADR, i, j);
        store(A, 0, i, j, C, Jd, true);
    }
    if (j < nth) {
        // D^theta at (i, j+1/2)
        T C = (X.Hph(i - 1, j) - X.Hph(i, j)) * X.t(T_INV_ADT, i, j);
        T Jd = __ldg(A.J[1] + qf) * X.t(T_INV_ADT, i, j);
        store(A, 1, i, j, C, Jd, false);
        // B^r at (i, j+1/2)
        T Cb = -(X.Eph(i, j + 1) - X.Eph(i, j)) * X.t(T_INV_ABR, i, j);
        store(A, 3, i, j, Cb, T(0), false);
    }
    if (j > 0 && j < nth) {
        // D^phi at (i, j)
        T C = ((X.Hth(i, j) - X.Hth(i - 1, j)) * A.dth + (X.Hr(i, j - 1) - X.Hr(i, j)) * drd) * X.t(T_INV_ADP, i, j);
        T Jd = __ldg(A.J[2] + qf) * X.t(T_INV_ADP, i, j);
        store(A, 2, i, j, C, Jd, false);
        // B^theta at (i+1/2, j)
        if (i <= nr - 1) {
            T Cb = -(X.Eph(i, j) - X.Eph(i + 1, j)) * X.t(T_INV_ABT, i, j);
            store(A, 4, i, j, Cb, T(0), true);
        }
    } else {
        store_zero(A, 2, i, j, false);
        if (i <= nr - 1) store_zero(A, 4, i, j, true);
    }
    // B^phi at (i+1/2, j+1/2)
    if (i <= nr - 1 && j < nth) {
        T C = -((X.Eth(i + 1, j) - X.Eth(i, j)) * A.dth + (X.Er(i, j) - X.Er(i, j + 1)) * drp) * X.t(T_INV_ABP, i, j);
        store(A, 5, i, j, C, T(0), true);
    }
    (void)qt;
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
    return run_field<float>(ctx, f, ctx->tab32, ctx->col1d32, s, j_lo, j_hi);
}

}  // namespace grpic
