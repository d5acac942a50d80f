// grpic_diag.cu -- diagnostics of Sec. 3.4 of arXiv:2503.04558: the vertex
// charge density rho = sum q w S / dV (cloud in cell, dV = A^D_phi with
// dphi = 1) and the discrete div D in the integral form of Eq. J-integral-eqn,
// whose difference must stay at round-off under the charge-conserving
// deposit.  Also the standalone deposit entry (moves given by two particle
// states and their azimuthal displacement).
#include "grpic_internal.cuh"
#include "grpic_shape3.cuh"

namespace grpic {
namespace {

__device__ __forceinline__ int jcl(const GridDev &g, double x2)
{
    int j = (int)floor(x2);
    return j > g.nth - 1 ? g.nth - 1 : j;
}

template <typename T>
__device__ __forceinline__ void logical(const GridDev &g, const void *x1, const void *x2, const int32_t *cell, int64_t p,
                                        double &a, double &b)
{
    if (sizeof(T) == 8) {
        a = (log(((const double *)x1)[p]) - g.ln_rin) / g.dx1;
        b = ((const double *)x2)[p] / g.dth;
    } else {
        // FP32 form: cell key and offsets; the last row holds the distance
        // to theta = pi
        int c = cell[p];
        a = (c % g.nr) + (double)((const float *)x1)[p];
        const int j = c / g.nr;
        const double o = (double)((const float *)x2)[p];
        b = (j == g.nth - 1) ? (double)g.nth - o : j + o;
    }
}

// T: the particle and field precision of the context; A: the type rho and
// div D are accumulated and stored in (T for the diagnostics, double for the
// charge check)
template <typename T, typename A = T>
__global__ void rho_particles(GridDev g, int64_t nmax, const int64_t *d_count, const void *x1, const void *x2,
                              const int32_t *cell, const uint32_t *tag, const double *qw, A *rho, int64_t ld,
                              int shape)
{
    int64_t n = d_count ? *d_count : nmax;
    if (n > nmax) n = nmax;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t t = tag[p];
    if (t & DEAD) return;
    double a, b;
    logical<T>(g, x1, x2, cell, p, a, b);
    if (!(a >= -1.0 && a < g.nr + 1.0 && b >= 0.0 && b <= (double)g.nth)) return;  // outside the arrays
    if (shape == 3) {
        // cubic weights on the 4 x 4 vertices, rows past the axis folded
        // (even), columns past the guard columns dropped
        const int i = (int)floor(a), j = (int)floor(b);
        const double q = qw[t & 3u];
        for (int ka = -1; ka <= 2; ++ka) {
            const int k = i + ka;
            if (k < -NG || k > g.nr + NG - 1) continue;
            const double wr = w3(a - k);
            for (int lb = -1; lb <= 2; ++lb) {
                bool flip;
                const int l = mirror_row(j + lb, false, g.nth, flip);
                atomicAdd(rho + (size_t)l * ld + k + NG, (A)(q * wr * w3(b - (j + lb))));
            }
        }
        return;
    }
    int i = (int)floor(a), j = jcl(g, b);
    double f = a - i, h = b - j, q = qw[t & 3u];
    A *r0 = rho + (size_t)j * ld + i + NG;
    A *r1 = r0 + ld;
    atomicAdd(r0, (A)(q * (1 - f) * (1 - h)));
    atomicAdd(r0 + 1, (A)(q * f * (1 - h)));
    atomicAdd(r1, (A)(q * (1 - f) * h));
    atomicAdd(r1 + 1, (A)(q * f * h));
}

template <typename T, typename A = T>
__global__ void vertex_diag(GridDev g, const double *tab, size_t slab, const T *D0, const T *D1, A *rho, A *divD,
                            int64_t ld)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (col >= g.ld_tab || j > g.nth) return;
    size_t q = (size_t)j * ld + col, qt = (size_t)j * g.ld_tab + col;
    double idv = tab[T_INV_ADP * slab + qt];
    if (rho) rho[q] = (A)((double)rho[q] * idv);
    if (col == 0) {
        divD[q] = (A)0;
        return;
    }
    double flux = (double)D0[q] * tab[T_ADR * slab + qt] - (double)D0[q - 1] * tab[T_ADR * slab + qt - 1];
    if (j < g.nth) flux += (double)D1[q] * tab[T_ADT * slab + qt];
    if (j > 0) flux -= (double)D1[q - ld] * tab[T_ADT * slab + qt - g.ld_tab];
    divD[q] = (A)(flux * idv);
}

// max |div D - rho - base| and max |rho| over the interior vertices
// (columns imin..imax, all rows) into out[0], out[1] as the bit patterns of
// non-negative doubles (ordered like the integers); state = div D - rho
__global__ void charge_check_kernel(int imin, int imax, int nth, const double *rho, const double *divD,
                                    const double *base, double *state, int64_t ld, unsigned long long *out)
{
    __shared__ double sr[256], sq[256];
    double mres = 0.0, mrho = 0.0;
    const int w = imax - imin + 1;
    const int64_t n = (int64_t)w * (nth + 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int i = imin + (int)(e % w), j = (int)(e / w);
        size_t q = (size_t)j * ld + i + NG;
        double d = divD[q] - rho[q];
        if (state) state[q] = d;
        mres = fmax(mres, fabs(d - (base ? base[q] : 0.0)));
        mrho = fmax(mrho, fabs(rho[q]));
    }
    sr[threadIdx.x] = mres;
    sq[threadIdx.x] = mrho;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + o]);
            sq[threadIdx.x] = fmax(sq[threadIdx.x], sq[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(sr[0]));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(sq[0]));
    }
}

// deposit of given moves (FP64 state layout), same window algebra as the push
__device__ __forceinline__ double W1(double d)
{
    d = fabs(d);
    return d < 1.0 ? 1.0 - d : 0.0;
}

template <typename T>
__global__ void deposit_kernel(GridDev g, int64_t nmax, const void *xa1, const void *xa2, const int32_t *ca,
                               const void *xb1, const void *xb2, const int32_t *cb, const uint32_t *tag, const void *dphi,
                               const double *qw, double dt, T *J0, T *J1, T *J2, int64_t ld, int *status,
                               int shape)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nmax) return;
    uint32_t t = tag[p];
    if (t & DEAD) return;
    double x1a, x2a, x1b, x2b;
    logical<T>(g, xa1, xa2, ca, p, x1a, x2a);
    logical<T>(g, xb1, xb2, cb, p, x1b, x2b);
    double dp = (sizeof(T) == 8) ? ((const double *)dphi)[p] : (double)((const float *)dphi)[p];
    if (!(isfinite(x1a) && isfinite(x2a) && isfinite(x1b) && isfinite(x2b) && isfinite(dp))) {
        set_status(status, GRPIC_ENAN);
        return;
    }
    // the 4x4 window (columns i0-1..i0+2) must stay inside the arrays
    if (!(x1a >= 0.0 && x1a < (double)g.nr && x2a >= 0.0 && x2a <= (double)g.nth && x2b >= 0.0 &&
          x2b <= (double)g.nth)) {
        set_status(status, GRPIC_ERANGE);
        return;
    }
    int i0 = (int)floor(x1a), j0 = jcl(g, x2a);
    int di = (int)floor(x1b) - i0, dj = jcl(g, x2b) - j0;
    if (di < -1 || di > 1 || dj < -1 || dj > 1) {
        set_status(status, GRPIC_ERANGE);
        return;
    }
    double q = qw[t & 3u];
    if (shape == 3) {
        if constexpr (sizeof(T) == 8)
            deposit3(g.nr, g.nth, ld, (double *)J0, (double *)J1, (double *)J2, q, dt, x1a, x2a, x1b, x2b, dp);
        return;
    }
    double S0r[4], S1r[4], S0t[4], S1t[4];
    for (int k = 0; k < 4; ++k) {
        S0r[k] = W1(x1a - (i0 - 1 + k));
        S1r[k] = W1(x1b - (i0 - 1 + k));
        S0t[k] = W1(x2a - (j0 - 1 + k));
        S1t[k] = W1(x2b - (j0 - 1 + k));
    }
    double cr = -q / (2.0 * dt), cp = q * dp / dt;
    double Pr = 0.0;
    for (int k = 0; k < 3; ++k) {
        Pr += S1r[k] - S0r[k];
        for (int l = 0; l < 4; ++l) {
            int row = j0 - 1 + l;
            double v = cr * Pr * (S1t[l] + S0t[l]);
            if (v != 0.0 && row >= 0 && row <= g.nth) atomicAdd(J0 + (size_t)row * ld + i0 - 1 + k + NG, (T)v);
        }
    }
    double Pt = 0.0;
    for (int l = 0; l < 3; ++l) {
        Pt += S1t[l] - S0t[l];
        int row = j0 - 1 + l;
        for (int k = 0; k < 4; ++k) {
            double v = cr * (S1r[k] + S0r[k]) * Pt;
            if (v != 0.0 && row >= 0 && row <= g.nth - 1) atomicAdd(J1 + (size_t)row * ld + i0 - 1 + k + NG, (T)v);
        }
    }
    for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) {
            int row = j0 - 1 + l;
            double v = cp * (S1r[k] * S1t[l] * (1.0 / 3.0) + S1r[k] * S0t[l] * (1.0 / 6.0) +
                             S0r[k] * S1t[l] * (1.0 / 6.0) + S0r[k] * S0t[l] * (1.0 / 3.0));
            if (v != 0.0 && row >= 0 && row <= g.nth) atomicAdd(J2 + (size_t)row * ld + i0 - 1 + k + NG, (T)v);
        }
}

template <typename T>
cudaError_t diag_t(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, void *rho, void *divD,
                   const double *d_qw, cudaStream_t s)
{
    size_t bytes = (size_t)(ctx->g.nth + 1) * f->ld * sizeof(T);
    if (rho) {
        cudaMemsetAsync(rho, 0, bytes, s);
        if (p && p->n > 0)
            rho_particles<T><<<(unsigned)((p->n + 255) / 256), 256, 0, s>>>(
                ctx->g, p->n, p->d_count, p->x1, p->x2, p->cell, p->tag, d_qw, (T *)rho, f->ld, ctx->prm.shape_order);
    }
    dim3 blk(32, 4), grd((ctx->g.ld_tab + 31) / 32, (ctx->g.nth + 1 + 3) / 4);
    vertex_diag<T><<<grd, blk, 0, s>>>(ctx->g, ctx->tab, ctx->slab, (const T *)f->D[0], (const T *)f->D[1], (T *)rho,
                                       (T *)divD, f->ld);
    return cudaGetLastError();
}

template <typename T>
cudaError_t check_t(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, double *rho, double *divD,
                    const double *base, double *state, unsigned long long *out, const double *d_qw, cudaStream_t s)
{
    size_t bytes = (size_t)(ctx->g.nth + 1) * f->ld * sizeof(double);
    cudaMemsetAsync(rho, 0, bytes, s);
    cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
    if (p && p->n > 0)
        rho_particles<T, double><<<(unsigned)((p->n + 255) / 256), 256, 0, s>>>(
            ctx->g, p->n, p->d_count, p->x1, p->x2, p->cell, p->tag, d_qw, rho, f->ld, ctx->prm.shape_order);
    dim3 blk(32, 4), grd((ctx->g.ld_tab + 31) / 32, (ctx->g.nth + 1 + 3) / 4);
    vertex_diag<T, double><<<grd, blk, 0, s>>>(ctx->g, ctx->tab, ctx->slab, (const T *)f->D[0], (const T *)f->D[1],
                                               rho, divD, f->ld);
    int imax = ctx->g.nr - ctx->grid.damp_cells - 1;
    if (imax > ctx->g.nr - 1) imax = ctx->g.nr - 1;
    // a particle absorbed just inside r_in still covers vertex 1 with the
    // cubic shape's cloud: the interior starts one column further in
    const int imin = ctx->prm.shape_order == 3 ? 2 : 1;
    if (imax >= imin)
        charge_check_kernel<<<256, 256, 0, s>>>(imin, imax, ctx->g.nth, rho, divD, base, state, f->ld, out);
    return cudaGetLastError();
}

// FP64 (r, theta) <-> the FP32 form's (cell, o1, o2), in FP64
__global__ void encode32_kernel(GridDev g, int64_t n, const double *r, const double *th, int32_t *cell, float *o1,
                                float *o2)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double x1 = (log(r[p]) - g.ln_rin) / g.dx1, x2 = th[p] / g.dth;
    int i = (int)floor(x1), j = (int)floor(x2);
    i = i < 0 ? 0 : (i > g.nr - 1 ? g.nr - 1 : i);
    j = j < 0 ? 0 : (j > g.nth - 1 ? g.nth - 1 : j);
    cell[p] = j * g.nr + i;
    o1[p] = (float)(x1 - i);
    o2[p] = (float)(j == g.nth - 1 ? (double)g.nth - x2 : x2 - j);
}

__global__ void decode32_kernel(GridDev g, int64_t n, const int32_t *cell, const float *o1, const float *o2, double *r,
                                double *th)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int c = cell[p], j = c / g.nr, i = c - j * g.nr;
    const double x2 = j == g.nth - 1 ? (double)g.nth - (double)o2[p] : j + (double)o2[p];
    r[p] = g.r_in * exp((i + (double)o1[p]) * g.dx1);
    th[p] = x2 * g.dth;
}

}  // namespace

cudaError_t launch_charge_check(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, double *rho,
                                double *divD, const double *base, double *state, unsigned long long *out, cudaStream_t s)
{
    const double *d_qw = (const double *)(ctx->d_status + 4);
    if (ctx->prm.precision == 64) return check_t<double>(ctx, p, f, rho, divD, base, state, out, d_qw, s);
    return check_t<float>(ctx, p, f, rho, divD, base, state, out, d_qw, s);
}

// q*w per species lives in a tiny device array owned by the context's scratch
cudaError_t launch_diag(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, void *rho, void *divD,
                        cudaStream_t s)
{
    const double *d_qw = (const double *)(ctx->d_status + 4);
    if (ctx->prm.precision == 64) return diag_t<double>(ctx, p, f, rho, divD, d_qw, s);
    return diag_t<float>(ctx, p, f, rho, divD, d_qw, s);
}

cudaError_t launch_deposit(grpic_ctx *ctx, const grpic_particles *b, const grpic_particles *a, const void *dphi,
                           grpic_fields *f, cudaStream_t s)
{
    if (b->n <= 0) return cudaSuccess;
    const double *d_qw = (const double *)(ctx->d_status + 4);
    unsigned blocks = (unsigned)((b->n + 255) / 256);
    if (ctx->prm.precision == 64)
        deposit_kernel<double><<<blocks, 256, 0, s>>>(ctx->g, b->n, b->x1, b->x2, b->cell, a->x1, a->x2, a->cell,
                                                      a->tag, dphi, d_qw, ctx->prm.dt, (double *)f->J[0],
                                                      (double *)f->J[1], (double *)f->J[2], f->ld, ctx->d_status,
                                                      ctx->prm.shape_order);
    else
        deposit_kernel<float><<<blocks, 256, 0, s>>>(ctx->g, b->n, b->x1, b->x2, b->cell, a->x1, a->x2, a->cell, a->tag,
                                                     dphi, d_qw, ctx->prm.dt, (float *)f->J[0], (float *)f->J[1],
                                                     (float *)f->J[2], f->ld, ctx->d_status, 1);
    return cudaGetLastError();
}

}  // namespace grpic

extern "C" grpic_status grpic_fp32_encode(grpic_ctx *ctx, int64_t n, const double *r, const double *theta,
                                          int32_t *cell, float *o1, float *o2, void *stream)
{
    using namespace grpic;
    if (!ctx || n < 0 || (n > 0 && (!r || !theta || !cell || !o1 || !o2))) return GRPIC_EINVAL;
    if (n == 0) return GRPIC_OK;
    encode32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(ctx->g, n, r, theta, cell, o1, o2);
    return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}

extern "C" grpic_status grpic_fp32_decode(grpic_ctx *ctx, int64_t n, const int32_t *cell, const float *o1,
                                          const float *o2, double *r, double *theta, void *stream)
{
    using namespace grpic;
    if (!ctx || n < 0 || (n > 0 && (!r || !theta || !cell || !o1 || !o2))) return GRPIC_EINVAL;
    if (n == 0) return GRPIC_OK;
    decode32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(ctx->g, n, cell, o1, o2, r, theta);
    return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ECUDA;
}
