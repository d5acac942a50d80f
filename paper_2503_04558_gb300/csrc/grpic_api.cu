// grpic_api.cu -- the extern "C" boundary declared in include/grpic.h.
// Argument checking, context (tables + scratch) management and the order of
// the per-step kernels (Fig. stepping of arXiv:2503.04558: push with deposit,
// field update, then the sort by cell).
#include "grpic_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>

using namespace grpic;

namespace {

grpic_status fail(grpic_ctx *ctx, grpic_status st, const char *msg)
{
    if (ctx) snprintf(ctx->err, sizeof ctx->err, "%s", msg);
    return st;
}

grpic_status cuda_fail(grpic_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) snprintf(ctx->err, sizeof ctx->err, "%s: %s", where, cudaGetErrorString(e));
    return GRPIC_ECUDA;
}

// Gauss-Legendre nodes/weights on [-1,1]: roots of P_n by Newton iteration on
// the three-term recurrence (the textbook construction).
void gauss_legendre(int n, double *x, double *w)
{
    for (int k = 0; k < n; ++k) {
        double z = std::cos(M_PI * (k + 0.75) / (n + 0.5));
        double pn = 0.0, dpn = 1.0;
        for (int iter = 0; iter < 64; ++iter) {
            double pm1 = 1.0, p = z;
            for (int l = 2; l <= n; ++l) {
                double pp = ((2 * l - 1) * z * p - (l - 1) * pm1) / l;
                pm1 = p;
                p = pp;
            }
            pn = p;
            dpn = n * (z * pn - pm1) / (z * z - 1.0);
            double step = pn / dpn;
            z -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double pm1 = 1.0, p = z;
        for (int l = 2; l <= n; ++l) {
            double pp = ((2 * l - 1) * z * p - (l - 1) * pm1) / l;
            pm1 = p;
            p = pp;
        }
        dpn = n * (z * p - pm1) / (z * z - 1.0);
        x[k] = z;
        w[k] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

__global__ void to_float(const double *a, float *b, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

cudaStream_t S(void *stream) { return (cudaStream_t)stream; }

bool fields_ok(const grpic_ctx *ctx, const grpic_fields *f)
{
    if (!f || f->ld < ctx->g.nr + 2 * NG) return false;
    if ((int64_t)(ctx->g.nth + 1) * f->ld > INT32_MAX) return false;  // element offsets are 32-bit
    for (int k = 0; k < 3; ++k)
        if (!f->D[k] || !f->B[k] || !f->J[k]) return false;
    return true;
}

bool particles_ok(const grpic_ctx *ctx, const grpic_particles *p)
{
    if (!p || p->n < 0 || p->capacity < p->n) return false;
    if (p->n == 0) return true;
    if (!p->x1 || !p->x2 || !p->u1 || !p->u2 || !p->u3 || !p->tag) return false;
    if (ctx->prm.precision == 32 && !p->cell) return false;
    if (p->n > INT32_MAX) return false;  // slot indices of the sort are int32
    return true;
}

size_t fsize(const grpic_ctx *ctx) { return ctx->prm.precision == 64 ? sizeof(double) : sizeof(float); }

grpic_status ensure_field_scratch(grpic_ctx *ctx, int64_t ld)
{
    static_assert(sizeof(int64_t) == 8, "");
    // 18 arrays: C^n (6) and two iterate buffers (12), stride ld; in the
    // FP32 form also the push's stencil quads of the six components
    size_t need = 18 * (size_t)(ctx->g.nth + 1) * (size_t)ld * fsize(ctx);
    size_t qneed = ctx->prm.precision == 32 ? 6 * (size_t)(ctx->g.nth + 1) * (size_t)ld * 16 : 0;
    if (ctx->fscratch && ctx->fscratch_ld == ld) return GRPIC_OK;
    if (ctx->fscratch) cudaFree(ctx->fscratch);
    if (ctx->q32) cudaFree(ctx->q32);
    ctx->fscratch = ctx->q32 = nullptr;
    ctx->fscratch_ld = 0;
    cudaError_t e = cudaMalloc(&ctx->fscratch, need);
    if (e == cudaSuccess && qneed) e = cudaMalloc(&ctx->q32, qneed);
    if (e != cudaSuccess) {
        if (ctx->fscratch) cudaFree(ctx->fscratch);
        ctx->fscratch = ctx->q32 = nullptr;
        return fail(ctx, GRPIC_ENOMEM, "field scratch allocation failed");
    }
    cudaMemset(ctx->fscratch, 0, need);
    ctx->fscratch_ld = ld;
    return GRPIC_OK;
}

// Ahead of each push on stream s: J zeroed and, if cnt9 is given, the 9 x
// n_cells direction counts of the next neighbour sort zeroed; in the FP32
// form one kernel does both while it rebuilds the push's view of the fields,
// their stencil quads, from D and B (the FP64 push reads the arrays).
grpic_status prepare_push(grpic_ctx *ctx, grpic_fields *f, int32_t *cnt9, cudaStream_t s)
{
    if (ctx->prm.precision != 32) {
        const size_t bytes = (size_t)(ctx->g.nth + 1) * f->ld * fsize(ctx);
        for (int k = 0; k < 3; ++k) cudaMemsetAsync(f->J[k], 0, bytes, s);
        if (cnt9) cudaMemsetAsync(cnt9, 0, sizeof(int32_t) * 9 * (size_t)ctx->g.nr * ctx->g.nth, s);
        return GRPIC_OK;
    }
    grpic_status st = ensure_field_scratch(ctx, f->ld);
    if (st) return st;
    cudaError_t e = launch_quad32(ctx, f, true, cnt9, s);
    return e == cudaSuccess ? GRPIC_OK : cuda_fail(ctx, e, "field quads");
}

grpic_status ensure_particle_scratch(grpic_ctx *ctx, int64_t n)
{
    if (n <= ctx->keys_cap) return GRPIC_OK;
    if (ctx->d_keys) cudaFree(ctx->d_keys);
    if (ctx->d_perm) cudaFree(ctx->d_perm);
    ctx->d_keys = nullptr;
    ctx->d_perm = nullptr;
    ctx->keys_cap = 0;
    if (cudaMalloc(&ctx->d_keys, sizeof(int32_t) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&ctx->d_perm, sizeof(int32_t) * (size_t)n) != cudaSuccess)
        return fail(ctx, GRPIC_ENOMEM, "particle scratch allocation failed");
    ctx->keys_cap = n;
    ctx->perm_cap = n;
    return GRPIC_OK;
}

// materialize = false (inside grpic_step, a push follows): the order is left
// in ctx->d_perm and the next push reads the particles through it
grpic_status sort_impl(grpic_ctx *ctx, grpic_particles *p, grpic_particles *q, cudaStream_t s,
                       bool materialize = true)
{
    int64_t ncell = (int64_t)ctx->g.nr * ctx->g.nth;
    grpic_status st = ensure_particle_scratch(ctx, p->n);
    if (st) return st;
    if (!(ctx->keys_valid && ctx->keys_tag == p->tag)) {
        cudaMemsetAsync(ctx->d_count, 0, sizeof(int32_t) * (ncell + 1), s);
        cudaError_t e = launch_keys(ctx, p, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "keys");
        ctx->keys_valid = 1;
        ctx->hist_valid = 1;
        ctx->keys_tag = p->tag;
    }
    // the neighbour sort needs the particles to be the last sort's output
    // with exactly one push since (the device re-checks the rest)
    bool neighbour = p->n > 0 && p->tag && ctx->sorted_tag == p->tag && ctx->pushes_since_sort == 1;
    if (!neighbour && !ctx->hist_valid) {
        cudaMemsetAsync(ctx->d_count, 0, sizeof(int32_t) * (ncell + 1), s);
        cudaError_t e = launch_hist(ctx, p, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "histogram");
        ctx->hist_valid = 1;
    }
    const bool counts_ready = neighbour && ctx->counts_ready;
    ctx->counts_ready = 0;
    cudaError_t e = launch_sort_step(ctx, p, q, neighbour, !ctx->hist_valid, materialize, counts_ready, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sort");
    ctx->keys_valid = 0;
    ctx->hist_valid = 0;
    std::swap(ctx->d_offset, ctx->d_offset_prev);  // segments of the new order
    if (!materialize) {
        ctx->pending_perm = 1;
        ctx->pending_tag = p->tag;
        return GRPIC_OK;
    }
    // the sorted state now lives in q's arrays: swap the array pointers
    std::swap(p->x1, q->x1);
    std::swap(p->x2, q->x2);
    std::swap(p->u1, q->u1);
    std::swap(p->u2, q->u2);
    std::swap(p->u3, q->u3);
    std::swap(p->tag, q->tag);
    std::swap(p->cell, q->cell);
    ctx->sorted_tag = p->tag;
    ctx->pushes_since_sort = 0;
    return GRPIC_OK;
}

grpic_status push_impl(grpic_ctx *ctx, grpic_particles *p, grpic_fields *f, bool for_sort, cudaStream_t s,
                       grpic_particles *scratch = nullptr)
{
    int64_t ncell = (int64_t)ctx->g.nr * ctx->g.nth;
    if (ctx->pending_perm) {
        // the last sort left its order in d_perm: read p through it and write
        // the pushed particles, in that order, into scratch's arrays
        if (!scratch || p->tag != ctx->pending_tag) return fail(ctx, GRPIC_EINVAL, "push: a sort's order is pending");
        // the counts of the next neighbour sort come from this push
        grpic_status fs = prepare_push(ctx, f, ctx->d_cnt9, s);
        if (fs) return fs;
        ctx->pending_perm = 0;
        grpic_particles out = *scratch;
        out.n = p->n;
        out.d_count = p->d_count;
        const int32_t *live = ctx->d_offset_prev + ncell;
        cudaError_t e = (ctx->prm.precision == 64)
                            ? launch_push64(ctx, p, &out, ctx->d_perm, live, ctx->d_cnt9, f, false, s)
                            : launch_push32(ctx, p, &out, ctx->d_perm, live, ctx->d_cnt9, f, false, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "push");
        ctx->counts_ready = 1;
        std::swap(p->x1, scratch->x1);
        std::swap(p->x2, scratch->x2);
        std::swap(p->u1, scratch->u1);
        std::swap(p->u2, scratch->u2);
        std::swap(p->u3, scratch->u3);
        std::swap(p->tag, scratch->tag);
        std::swap(p->cell, scratch->cell);
        // p now holds the sorted order pushed once: the next sort is a neighbour sort
        ctx->sorted_tag = p->tag;
        ctx->pushes_since_sort = 1;
        ctx->keys_valid = 1;
        ctx->hist_valid = 0;
        ctx->keys_tag = p->tag;
        return GRPIC_OK;
    }
    // the histogram serves the general sort only: a sort that will be a
    // neighbour sort rebuilds it from the keys if the device falls back
    const bool neighbour_next = p->n > 0 && p->tag && p->tag == ctx->sorted_tag && ctx->pushes_since_sort == 0;
    const bool histogram = for_sort && !neighbour_next;
    grpic_status st = ensure_particle_scratch(ctx, p->n);
    if (!st) st = prepare_push(ctx, f, nullptr, s);
    if (st) return st;
    if (histogram) cudaMemsetAsync(ctx->d_count, 0, sizeof(int32_t) * (ncell + 1), s);
    ctx->counts_ready = 0;
    cudaError_t e = (ctx->prm.precision == 64) ? launch_push64(ctx, p, p, nullptr, nullptr, nullptr, f, histogram, s)
                                                : launch_push32(ctx, p, p, nullptr, nullptr, nullptr, f, histogram, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "push");
    ctx->keys_valid = 1;  // the push writes every slot's key
    ctx->hist_valid = histogram ? 1 : 0;
    ctx->keys_tag = p->tag;
    ctx->pushes_since_sort = (p->tag == ctx->sorted_tag) ? ctx->pushes_since_sort + 1 : 2;
    return GRPIC_OK;
}

grpic_status field_impl(grpic_ctx *ctx, grpic_fields *f, cudaStream_t s)
{
    grpic_status st = ensure_field_scratch(ctx, f->ld);
    if (st) return st;
    cudaError_t e = (ctx->prm.precision == 64) ? launch_field64(ctx, f, s) : launch_field32(ctx, f, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "field update");
    return GRPIC_OK;
}

// scratch for the adjoint translation unit (same buffers as the step's)
}  // namespace

grpic_status grpic::ensure_field_scratch_ext(grpic_ctx *ctx, int64_t ld) { return ensure_field_scratch(ctx, ld); }
grpic_status grpic::ensure_particle_scratch_ext(grpic_ctx *ctx, int64_t n) { return ensure_particle_scratch(ctx, n); }

namespace {

// halo add: f[k] rows [row0, row0 + nrows) += buf (component-major, rows
// contiguous as in the field arrays); the component pointers by value
template <typename T>
struct HaloComps {
    T *p[6];
};

template <typename T>
__global__ void halo_add_kernel(HaloComps<T> comp, int ncomp, size_t off, size_t n, const T *buf)
{
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)ncomp * n;
    for (; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const size_t k = q / n, e = q - k * n;
        comp.p[k][off + e] += buf[q];
    }
}

// the arrays of one particle buffer, with element sizes
int particle_arrays(const grpic_ctx *ctx, const grpic_particles *p, void *arr[7], size_t esz[7])
{
    size_t fs = fsize(ctx);
    void *a[7] = {p->x1, p->x2, p->u1, p->u2, p->u3, (void *)p->tag, (void *)p->cell};
    size_t e[7] = {fs, fs, fs, fs, fs, 4, 4};
    int na = ctx->prm.precision == 32 ? 7 : 6;
    for (int k = 0; k < na; ++k) {
        arr[k] = a[k];
        esz[k] = e[k];
    }
    return na;
}

// the sort's caches no longer describe a buffer that was written from outside
void drop_sort_state(grpic_ctx *ctx)
{
    ctx->keys_valid = 0;
    ctx->hist_valid = 0;
    ctx->sorted_tag = nullptr;
    ctx->keys_tag = nullptr;
    ctx->counts_ready = 0;
}

}  // namespace

extern "C" {

grpic_status grpic_init(grpic_metric metric, double spin, const grpic_grid *grid, const grpic_params *prm,
                        grpic_ctx **out)
{
    if (!out) return GRPIC_EINVAL;
    *out = nullptr;
    if (metric != GRPIC_METRIC_KERR_SCHILD || !grid || !prm) return GRPIC_EINVAL;
    if (!(spin >= 0.0 && spin < 1.0)) return GRPIC_EINVAL;
    if (grid->n_r < 4 || grid->n_theta < 4 || (grid->n_theta & 1)) return GRPIC_EINVAL;
    if ((int64_t)grid->n_r * grid->n_theta > (int64_t)1 << 28) return GRPIC_EINVAL;
    if (!(grid->r_in > 0.0 && grid->r_out > grid->r_in)) return GRPIC_EINVAL;
    if (grid->damp_cells < 0 || grid->damp_cells > grid->n_r || !(grid->damp_max >= 0.0 && grid->damp_max <= 1.0))
        return GRPIC_EINVAL;
    if (!(prm->dt > 0.0) || prm->n_field_iter < 0 || prm->n_push_iter < 0 || prm->n_push_iter > 64 ||
        prm->n_field_iter > 64)
        return GRPIC_EINVAL;
    if (prm->precision != 64 && prm->precision != 32) return GRPIC_EINVAL;
    if (prm->island_arith != 0 && prm->island_arith != 1) return GRPIC_EINVAL;
    if (prm->pusher != 0 && prm->pusher != 1) return GRPIC_EINVAL;
    if (!(prm->shape_order == 1 || (prm->shape_order == 3 && prm->precision == 64))) return GRPIC_EINVAL;
    if ((prm->radiation != 0 && prm->radiation != 1) || (prm->injection != 0 && prm->injection != 1) ||
        ((prm->radiation || prm->injection) && prm->precision != 64))
        return GRPIC_EINVAL;
    if (prm->radiation && !(prm->eps_ph > 0.0 && prm->gamma_thr >= 1.0 && prm->tau >= 0.0)) return GRPIC_EINVAL;
    if (prm->injection && !(prm->sigma_thr >= 0.0 && prm->eps_db >= 0.0)) return GRPIC_EINVAL;
    if (!(prm->beta_field >= 0.0 && prm->beta_field <= 1.0)) return GRPIC_EINVAL;

    grpic_ctx *ctx = new (std::nothrow) grpic_ctx();
    if (!ctx) return GRPIC_ENOMEM;
    memset((void *)ctx, 0, sizeof *ctx);
    cudaGetDevice(&ctx->device);
    ctx->grid = *grid;
    ctx->prm = *prm;
    ctx->field_fused = 1;
    GridDev &g = ctx->g;
    g.nr = grid->n_r;
    g.nth = grid->n_theta;
    g.ld_tab = grid->n_r + 2 * NG;
    g.a = spin;
    g.r_in = grid->r_in;
    g.r_out = grid->r_out;
    g.dx1 = std::log(grid->r_out / grid->r_in) / grid->n_r;
    g.dth = M_PI / grid->n_theta;
    g.ln_rin = std::log(grid->r_in);
    gauss_legendre(NGL, ctx->gl_x, ctx->gl_w);
    ctx->slab = (size_t)(g.nth + 1) * g.ld_tab;
    int64_t ncell = (int64_t)g.nr * g.nth;

    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&ctx->tab, sizeof(double) * ctx->slab * T_COUNT);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->col1d, sizeof(double) * 4 * g.ld_tab);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 64);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_count, sizeof(int32_t) * (ncell + 2));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_offset, sizeof(int32_t) * (ncell + 3));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_cursor, sizeof(int32_t) * (ncell + 3));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_blocksum, sizeof(int32_t) * 8192);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_bigseg, sizeof(int32_t) * (ncell + 1));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_offset_prev, sizeof(int32_t) * (ncell + 3));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_cnt9, sizeof(int32_t) * 9 * ncell);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_base9, sizeof(int32_t) * 9 * ncell);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_sortflag, sizeof(int32_t));
    if (e == cudaSuccess) {
        e = cudaMalloc(&ctx->rcol, sizeof(double) * g.ld_tab);
        if (e == cudaSuccess) {
            double *h = (double *)malloc(sizeof(double) * g.ld_tab);
            for (int c = 0; c < g.ld_tab; ++c) h[c] = g.r_in * std::exp((c - NG) * g.dx1);
            e = cudaMemcpy(ctx->rcol, h, sizeof(double) * g.ld_tab, cudaMemcpyHostToDevice);
            free(h);
        }
    }
    if (e != cudaSuccess) {
        grpic_destroy(ctx);
        return GRPIC_ENOMEM;
    }
    cudaMemset(ctx->d_status, 0, 64);
    cudaMemset(ctx->d_offset_prev, 0, sizeof(int32_t) * (ncell + 3));  // no segments before the first sort
    // q*w per species next to the status word (read by the diagnostics)
    cudaMemcpy((char *)ctx->d_status + 16, prm->q_weight, 4 * sizeof(double), cudaMemcpyHostToDevice);
    e = launch_tables(ctx, 0);
    if (e == cudaSuccess) e = sort_setup();
    if (e == cudaSuccess && (prm->radiation || prm->injection)) {
        e = cudaMalloc(&ctx->d_spqm, 4 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_spmassive, 4 * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_spqm, prm->q_over_m, 4 * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(ctx->d_spmassive, prm->massive, 4 * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && prm->precision == 32) {
        e = cudaMalloc(&ctx->tab32, sizeof(float) * ctx->slab * T_COUNT);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->col1d32, sizeof(float) * 4 * g.ld_tab);
        if (e == cudaSuccess) {
            size_t n = ctx->slab * T_COUNT;
            to_float<<<(unsigned)((n + 255) / 256), 256>>>(ctx->tab, ctx->tab32, n);
            to_float<<<(unsigned)((4 * g.ld_tab + 255) / 256), 256>>>(ctx->col1d, ctx->col1d32, 4 * g.ld_tab);
            e = cudaGetLastError();
        }
        // float-pair tables of the near-horizon island: r_i and sin/cos theta_j
        if (e == cudaSuccess) e = cudaMalloc(&ctx->rcol2, sizeof(float) * 2 * g.ld_tab);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->rowsc, sizeof(float) * 4 * (g.nth + 1));
        if (e == cudaSuccess) {
            auto split = [](double x, float *o) {
                o[0] = (float)x;
                o[1] = (float)(x - (double)o[0]);
            };
            float *h2 = (float *)malloc(sizeof(float) * 2 * g.ld_tab);
            float *h4 = (float *)malloc(sizeof(float) * 4 * (g.nth + 1));
            for (int c = 0; c < g.ld_tab; ++c) split(g.r_in * std::exp((c - NG) * g.dx1), h2 + 2 * c);
            for (int j = 0; j <= g.nth; ++j) {
                split(std::sin(j * g.dth), h4 + 4 * j);
                split(std::cos(j * g.dth), h4 + 4 * j + 2);
            }
            e = cudaMemcpy(ctx->rcol2, h2, sizeof(float) * 2 * g.ld_tab, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(ctx->rowsc, h4, sizeof(float) * 4 * (g.nth + 1), cudaMemcpyHostToDevice);
            free(h2);
            free(h4);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        grpic_destroy(ctx);
        return GRPIC_ECUDA;
    }
    *out = ctx;
    return GRPIC_OK;
}

grpic_status grpic_init_fields(grpic_ctx *ctx, grpic_field_kind kind, double B0, grpic_fields *f, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f) || kind < GRPIC_FIELD_WALD || kind > GRPIC_FIELD_SPLIT_MONOPOLE)
        return fail(ctx, GRPIC_EINVAL, "grpic_init_fields: bad fields or kind");
    cudaError_t e = launch_init_fields(ctx, (int)kind, B0, f, S(stream));
    return e == cudaSuccess ? GRPIC_OK : cuda_fail(ctx, e, "init_fields");
}

grpic_status grpic_push(grpic_ctx *ctx, grpic_particles *p, grpic_fields *f, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!particles_ok(ctx, p) || !fields_ok(ctx, f)) return fail(ctx, GRPIC_EINVAL, "grpic_push: bad arguments");
    return push_impl(ctx, p, f, true, S(stream));
}

grpic_status grpic_deposit(grpic_ctx *ctx, const grpic_particles *before, const grpic_particles *after,
                           const void *dphi, grpic_fields *f, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!particles_ok(ctx, before) || !particles_ok(ctx, after) || !fields_ok(ctx, f) || before->n != after->n ||
        (before->n > 0 && !dphi))
        return fail(ctx, GRPIC_EINVAL, "grpic_deposit: bad arguments");
    cudaError_t e = launch_deposit(ctx, before, after, dphi, f, S(stream));
    return e == cudaSuccess ? GRPIC_OK : cuda_fail(ctx, e, "deposit");
}

grpic_status grpic_field_update(grpic_ctx *ctx, grpic_fields *f, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f)) return fail(ctx, GRPIC_EINVAL, "grpic_field_update: bad fields");
    return field_impl(ctx, f, S(stream));
}

grpic_status grpic_sort(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!particles_ok(ctx, p) || !particles_ok(ctx, scratch) || scratch->capacity < p->n)
        return fail(ctx, GRPIC_EINVAL, "grpic_sort: bad arguments");
    return sort_impl(ctx, p, scratch, S(stream));
}

// one step: push (through a pending permutation if the last sort left one),
// field update, and the sort when due; materialize = false leaves the sort's
// order pending for the next step's push
static cudaEvent_t *timing_slot(grpic_ctx *ctx)
{
    if (!ctx->timing) return nullptr;
    if (!ctx->tevents) ctx->tevents = new std::vector<cudaEvent_t>();
    std::vector<cudaEvent_t> &v = *ctx->tevents;
    const size_t need = 4 * (size_t)(ctx->tsteps + 1);
    while (v.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        v.push_back(e);
    }
    return &v[4 * (size_t)ctx->tsteps];
}

static grpic_status step_one(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f,
                             bool materialize, cudaStream_t s, bool timed = true)
{
    const int every = ctx->prm.sort_every;
    const bool sort_now = every > 0 && ((ctx->step_count + 1) % every == 0);
    cudaEvent_t *ev = timed ? timing_slot(ctx) : nullptr;
    if (ev) cudaEventRecord(ev[0], s);
    grpic_status st = push_impl(ctx, p, f, sort_now, s, scratch);
    if (ev) cudaEventRecord(ev[1], s);
    if (!st) st = field_impl(ctx, f, s);
    if (ev) cudaEventRecord(ev[2], s);
    if (!st && sort_now) st = sort_impl(ctx, p, scratch, s, materialize);
    if (ev) {
        cudaEventRecord(ev[3], s);
        ctx->tsteps++;
    }
    if (!st) ctx->step_count++;
    return st;
}

// a failed call leaves the particle data valid but unsorted
static grpic_status drop_pending(grpic_ctx *ctx, grpic_status st)
{
    if (st && ctx->pending_perm) {
        ctx->pending_perm = 0;
        ctx->sorted_tag = nullptr;
    }
    return st;
}

// one step with 2D radiation and/or injection: push (with the emission and
// conversion decisions), the children appended, field update, injection,
// and a general sort that moves the data (the appends break the neighbour
// sort's precondition)
static grpic_status step_one_rad(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f,
                                 cudaStream_t s)
{
    cudaEvent_t *ev = timing_slot(ctx);
    if (ev) cudaEventRecord(ev[0], s);
    grpic_status st = push_impl(ctx, p, f, false, s);
    cudaError_t e = cudaSuccess;
    if (!st && ctx->prm.radiation) e = launch_append_children(ctx, p, s);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "radiation");
    if (ev) cudaEventRecord(ev[1], s);
    if (!st) st = field_impl(ctx, f, s);
    if (!st && ctx->prm.injection) {
        e = launch_injection(ctx, p, f, s);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "injection");
    }
    if (ev) cudaEventRecord(ev[2], s);
    if (!st) {
        ctx->hist_valid = 0;        // the appended slots carry keys, the histogram is rebuilt
        ctx->sorted_tag = nullptr;  // general path
        st = sort_impl(ctx, p, scratch, s, true);
    }
    if (ev) {
        cudaEventRecord(ev[3], s);
        ctx->tsteps++;
    }
    if (!st) ctx->step_count++;
    return st;
}

grpic_status grpic_step(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f, int nsteps,
                        void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    int every = ctx->prm.sort_every;
    if (nsteps < 0 || !particles_ok(ctx, p) || !fields_ok(ctx, f) ||
        (every > 0 && (!particles_ok(ctx, scratch) || scratch->capacity < p->n)))
        return fail(ctx, GRPIC_EINVAL, "grpic_step: bad arguments");
    if (ctx->prm.radiation || ctx->prm.injection) {
        // new particles: the whole capacity is the slot range, the device
        // count the live particles; every step sorts
        if (every != 1 || scratch->capacity < p->capacity)
            return fail(ctx, GRPIC_EINVAL, "grpic_step: radiation and injection need sort_every 1 and equal buffers");
        p->n = p->capacity;
        scratch->n = scratch->capacity;
        grpic_status st = ensure_particle_scratch(ctx, p->capacity);
        if (!st && ensure_rad_scratch(ctx, p->capacity) != cudaSuccess) st = fail(ctx, GRPIC_ENOMEM, "radiation scratch");
        for (int k = 0; k < nsteps && !st; ++k) st = step_one_rad(ctx, p, scratch, f, S(stream));
        return st;
    }
    grpic_status st = GRPIC_OK;
    // a sort followed by this call's next push leaves only its order (the
    // push reads through it); the call's last sort moves the data
    for (int k = 0; k < nsteps && !st; ++k) st = step_one(ctx, p, scratch, f, k == nsteps - 1, S(stream));
    return drop_pending(ctx, st);
}

// Steps 2 .. nsteps-1 of a run run as replays of a captured graph of two
// steps whose sorts leave their order pending (each push reads through the
// previous sort's permutation into the other buffer, so two steps bring the
// buffers back): the data moves once per call, in the last step's sort.
grpic_status grpic_step_graph(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f,
                              int nsteps, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (nsteps < 0 || ctx->prm.sort_every != 1 || !particles_ok(ctx, p) || !fields_ok(ctx, f) ||
        !particles_ok(ctx, scratch) || scratch->capacity < p->n)
        return fail(ctx, GRPIC_EINVAL, "grpic_step_graph: bad arguments (sort_every must be 1)");
    if (nsteps < 4 || ctx->prm.radiation || ctx->prm.injection) return grpic_step(ctx, p, scratch, f, nsteps, stream);
    grpic_status st = GRPIC_OK;
    int done = 0;
    // head: a plain step if the particles are not a sort's output, then one
    // step that leaves its sort pending
    if (!(ctx->sorted_tag == p->tag && ctx->pushes_since_sort == 0)) {
        st = step_one(ctx, p, scratch, f, true, S(stream));
        done++;
    }
    if (!st) {
        st = step_one(ctx, p, scratch, f, false, S(stream));
        done++;
    }
    const int steady = nsteps - done - 1;  // the last step materializes
    const int pairs = steady / 2;
    if (!st && pairs > 0) {
        const void *key[24] = {p->x1, p->x2, p->u1, p->u2, p->u3, p->tag, p->cell, p->d_count,
                               scratch->x1, scratch->x2, scratch->u1, scratch->u2, scratch->u3, scratch->tag,
                               scratch->cell, f->D[0], f->D[1], f->D[2], f->B[0], f->B[1], f->B[2], f->J[0], f->J[1],
                               f->J[2]};
        bool same = ctx->graph_exec && memcmp(key, ctx->graph_key, sizeof key) == 0 &&
                    ctx->keys_cap >= p->n && ctx->fscratch_ld == f->ld && ctx->graph_offset == ctx->d_offset;
        if (!same) {
            if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
            cudaError_t e = cudaSuccess;
            if (!ctx->cap_stream) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return drop_pending(ctx, cuda_fail(ctx, e, "graph stream"));
            // everything the two steps allocate is allocated already (the head
            // steps ran); the capture must wait for them
            st = ensure_particle_scratch(ctx, p->n);
            if (!st) st = ensure_field_scratch(ctx, f->ld);
            if (st) return drop_pending(ctx, st);
            cudaStreamSynchronize(S(stream));
            const int64_t sc = ctx->step_count;
            e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return drop_pending(ctx, cuda_fail(ctx, e, "graph capture"));
            st = step_one(ctx, p, scratch, f, false, ctx->cap_stream, false);
            if (!st) st = step_one(ctx, p, scratch, f, false, ctx->cap_stream, false);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(ctx->cap_stream, &g);
            ctx->step_count = sc;
            if (st || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return drop_pending(ctx, st ? st : cuda_fail(ctx, e, "graph capture"));
            }
            e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ctx->graph_exec = nullptr;
                return drop_pending(ctx, cuda_fail(ctx, e, "graph instantiate"));
            }
            memcpy(ctx->graph_key, key, sizeof key);
            ctx->graph_offset = ctx->d_offset;
            // the capture left the host bookkeeping of two steps: pointers, the
            // offsets' double buffer and the pending order as before them,
            // which is also the state after each replay
        }
        for (int k = 0; k < pairs; ++k) {
            cudaError_t e = cudaGraphLaunch(ctx->graph_exec, S(stream));
            if (e != cudaSuccess) return drop_pending(ctx, cuda_fail(ctx, e, "graph launch"));
            ctx->step_count += 2;
        }
        done += 2 * pairs;
    }
    while (!st && done < nsteps) {
        st = step_one(ctx, p, scratch, f, done == nsteps - 1, S(stream));
        done++;
    }
    return drop_pending(ctx, st);
}

// One step of grpic_step_host: the in-place push of push_impl over the slot
// range in chunks, chunk c launched once its copy in (event in[c]) has landed,
// then the field update and a sort that moves the data.
static grpic_status step_one_chunks(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f,
                                    int nch, int64_t chunk, const cudaEvent_t *in, cudaStream_t s)
{
    if (ctx->pending_perm) return fail(ctx, GRPIC_EINVAL, "grpic_step_host: a sort's order is pending");
    const int64_t ncell = (int64_t)ctx->g.nr * ctx->g.nth;
    const int every = ctx->prm.sort_every;
    const bool sort_now = every > 0 && ((ctx->step_count + 1) % every == 0);
    cudaEvent_t *ev = timing_slot(ctx);
    if (ev) cudaEventRecord(ev[0], s);
    const bool neighbour_next = p->n > 0 && p->tag && p->tag == ctx->sorted_tag && ctx->pushes_since_sort == 0;
    const bool histogram = sort_now && !neighbour_next;
    grpic_status st = ensure_particle_scratch(ctx, p->n);
    if (!st) st = prepare_push(ctx, f, nullptr, s);  // the fields are in place: s waited for their copy
    if (st) return st;
    if (histogram) cudaMemsetAsync(ctx->d_count, 0, sizeof(int32_t) * (ncell + 1), s);
    ctx->counts_ready = 0;
    const size_t es = ctx->prm.precision == 64 ? 8 : 4;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < nch && e == cudaSuccess; ++c) {
        const int64_t lo = c * chunk, hi = std::min(p->n, lo + chunk);
        e = cudaStreamWaitEvent(s, in[c], 0);
        grpic_particles q = *p;
        q.n = hi - lo;
        q.capacity = hi - lo;
        q.d_count = nullptr;
        q.x1 = static_cast<char *>(p->x1) + lo * es;
        q.x2 = static_cast<char *>(p->x2) + lo * es;
        q.u1 = static_cast<char *>(p->u1) + lo * es;
        q.u2 = static_cast<char *>(p->u2) + lo * es;
        q.u3 = static_cast<char *>(p->u3) + lo * es;
        q.tag = p->tag + lo;
        q.cell = p->cell ? p->cell + lo : nullptr;
        if (e == cudaSuccess)
            e = (ctx->prm.precision == 64) ? launch_push64(ctx, &q, &q, nullptr, nullptr, nullptr, f, histogram, s, lo)
                                           : launch_push32(ctx, &q, &q, nullptr, nullptr, nullptr, f, histogram, s, lo);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "push");
    ctx->keys_valid = 1;
    ctx->hist_valid = histogram ? 1 : 0;
    ctx->keys_tag = p->tag;
    ctx->pushes_since_sort = (p->tag == ctx->sorted_tag) ? ctx->pushes_since_sort + 1 : 2;
    if (ev) cudaEventRecord(ev[1], s);
    st = field_impl(ctx, f, s);
    if (ev) cudaEventRecord(ev[2], s);
    if (!st && sort_now) st = sort_impl(ctx, p, scratch, s, true);
    if (ev) {
        cudaEventRecord(ev[3], s);
        ctx->tsteps++;
    }
    if (!st) ctx->step_count++;
    return st;
}

// ---------------------------------------------------------------------------
// Steps with a host-resident particle state (grpic_step_host).  The slot range
// is cut into chunks; each step copies the chunks in on up_stream, runs one
// grpic_step on `stream`, reads the live count, and copies the chunks back
// on down_stream.  The next step's copy of chunk c in waits only for chunk
// c's copy out, so the two directions overlap.

}  // extern "C"

namespace {

__global__ void set_count_kernel(int64_t *d_count, int64_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_count = n;
}

constexpr int64_t HOST_CHUNK_MIN = int64_t(1) << 24;  // slots per chunk at least
constexpr int HOST_CHUNKS_MAX = 64;

struct HostArrays {
    void *a[7];
    size_t es[7];
    int n;
};

HostArrays host_arrays(const grpic_ctx *ctx, const grpic_particles *p)
{
    HostArrays h;
    const size_t e = ctx->prm.precision == 32 ? 4 : 8;
    void *ptrs[7] = {p->x1, p->x2, p->u1, p->u2, p->u3, p->tag, p->cell};
    size_t es[7] = {e, e, e, e, e, 4, 4};
    h.n = ctx->prm.precision == 32 ? 7 : 6;
    for (int k = 0; k < 7; ++k) {
        h.a[k] = ptrs[k];
        h.es[k] = es[k];
    }
    return h;
}

}  // namespace

extern "C" {

grpic_status grpic_step_host(grpic_ctx *ctx, grpic_particles *host, grpic_particles *dev, grpic_particles *dev_scratch,
                             const grpic_fields *host_f, grpic_fields *f, int nsteps, int64_t bytes[2], void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (bytes) bytes[0] = bytes[1] = 0;
    if (nsteps < 0 || !host || host->n < 0 || host->capacity < host->n || !particles_ok(ctx, dev) ||
        !particles_ok(ctx, dev_scratch) || !dev->d_count || dev->capacity < host->n ||
        dev_scratch->capacity < host->n || !fields_ok(ctx, f) || ctx->prm.radiation || ctx->prm.injection)
        return fail(ctx, GRPIC_EINVAL, "grpic_step_host: bad arguments");
    const HostArrays ha = host_arrays(ctx, host);
    for (int k = 0; k < ha.n; ++k)
        if (!ha.a[k] && host->n > 0) return fail(ctx, GRPIC_EINVAL, "grpic_step_host: missing host array");
    if (host_f) {
        if (host_f->ld != f->ld) return fail(ctx, GRPIC_EINVAL, "grpic_step_host: host fields' ld differs");
        for (int k = 0; k < 3; ++k)
            if (!host_f->D[k] || !host_f->B[k]) return fail(ctx, GRPIC_EINVAL, "grpic_step_host: missing host field");
    }
    cudaError_t e = cudaSuccess;
    if (!ctx->up_stream) e = cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->down_stream) e = cudaStreamCreateWithFlags(&ctx->down_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->h_count) e = cudaHostAlloc(reinterpret_cast<void **>(&ctx->h_count), sizeof(int64_t), 0);
    if (e == cudaSuccess && !ctx->hevents) {
        ctx->hevents = new (std::nothrow) std::vector<cudaEvent_t>();
        if (!ctx->hevents) return fail(ctx, GRPIC_ENOMEM, "grpic_step_host: events");
    }
    // events: [0, HOST_CHUNKS_MAX) chunks out, [HOST_CHUNKS_MAX, 2 HOST_CHUNKS_MAX)
    // chunks in, then fields out, fields in, step done, end
    const int nev = 2 * HOST_CHUNKS_MAX + 4;
    while (e == cudaSuccess && (int)ctx->hevents->size() < nev) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) ctx->hevents->push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "grpic_step_host: setup");
    std::vector<cudaEvent_t> &ev = *ctx->hevents;
    cudaEvent_t *ev_cin = ev.data() + HOST_CHUNKS_MAX;
    cudaEvent_t ev_fout = ev[2 * HOST_CHUNKS_MAX], ev_fin = ev[2 * HOST_CHUNKS_MAX + 1],
                ev_step = ev[2 * HOST_CHUNKS_MAX + 2], ev_end = ev[2 * HOST_CHUNKS_MAX + 3];
    cudaStream_t s = S(stream), up = ctx->up_stream, down = ctx->down_stream;
    const size_t fbytes = (size_t)(ctx->g.nth + 1) * f->ld * (ctx->prm.precision == 32 ? 4 : 8);
    int64_t n = host->n;
    int prev_chunks = 0;  // chunks copied out by the previous step
    int64_t prev_chunk = 0;
    grpic_status st = GRPIC_OK;
    // the copies in wait for the work already on `stream` (which may use the
    // device buffers) and for the previous call's copies out
    e = cudaEventRecord(ev_step, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(up, ev_step, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(up, ev_end, 0);
    for (int step = 0; step < nsteps && e == cudaSuccess && !st; ++step) {
        const int64_t chunk = std::max(HOST_CHUNK_MIN, (n + HOST_CHUNKS_MAX - 1) / HOST_CHUNKS_MAX);
        const int nch = n > 0 ? (int)((n + chunk - 1) / chunk) : 0;
        const HostArrays hd = host_arrays(ctx, dev);
        // copies in: the fields, then chunk c after the previous step's copy
        // out of the slots it covers; the push of a chunk waits for its copy
        if (host_f && e == cudaSuccess) {
            if (step > 0) e = cudaStreamWaitEvent(up, ev_fout, 0);
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                e = cudaMemcpyAsync(f->D[k], host_f->D[k], fbytes, cudaMemcpyHostToDevice, up);
                if (e == cudaSuccess) e = cudaMemcpyAsync(f->B[k], host_f->B[k], fbytes, cudaMemcpyHostToDevice, up);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_fin, up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_fin, 0);
        for (int c = 0; c < nch && e == cudaSuccess; ++c) {
            const int64_t lo = c * chunk, hi = std::min(n, lo + chunk);
            if (step > 0 && prev_chunks > 0) {
                const int last = (int)std::min<int64_t>(prev_chunks - 1, (hi - 1) / prev_chunk);
                for (int q = (int)(lo / prev_chunk); q <= last && e == cudaSuccess; ++q)
                    e = cudaStreamWaitEvent(up, ev[q], 0);
            }
            for (int k = 0; k < ha.n && e == cudaSuccess; ++k)
                e = cudaMemcpyAsync(static_cast<char *>(hd.a[k]) + lo * ha.es[k],
                                    static_cast<const char *>(ha.a[k]) + lo * ha.es[k], (hi - lo) * ha.es[k],
                                    cudaMemcpyHostToDevice, up);
            if (e == cudaSuccess) e = cudaEventRecord(ev_cin[c], up);
        }
        if (e != cudaSuccess) break;
        if (bytes) bytes[0] += n * (int64_t)(ha.n == 7 ? 28 : 44) + (host_f ? 6 * (int64_t)fbytes : 0);
        dev->n = n;
        set_count_kernel<<<1, 32, 0, s>>>(dev->d_count, n);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        st = step_one_chunks(ctx, dev, dev_scratch, f, nch, chunk, ev_cin, s);
        st = drop_pending(ctx, st);
        if (st) break;
        // the live count decides the copies out
        e = cudaMemcpyAsync(ctx->h_count, dev->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        const int64_t nn = std::min(*ctx->h_count, n);
        if (nn < 0) {
            st = fail(ctx, GRPIC_ECUDA, "grpic_step_host: bad live count");
            break;
        }
        e = cudaEventRecord(ev_step, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ev_step, 0);
        const int64_t ochunk = std::max(HOST_CHUNK_MIN, (nn + HOST_CHUNKS_MAX - 1) / HOST_CHUNKS_MAX);
        const int och = nn > 0 ? (int)((nn + ochunk - 1) / ochunk) : 0;
        const HostArrays hs = host_arrays(ctx, dev);  // the sorted state (dev swapped by the sort)
        // the fields first: the next step's copy in starts with them
        if (host_f && e == cudaSuccess) {
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                e = cudaMemcpyAsync(host_f->D[k], f->D[k], fbytes, cudaMemcpyDeviceToHost, down);
                if (e == cudaSuccess) e = cudaMemcpyAsync(host_f->B[k], f->B[k], fbytes, cudaMemcpyDeviceToHost, down);
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev_fout, down);
        }
        for (int c = 0; c < och && e == cudaSuccess; ++c) {
            const int64_t lo = c * ochunk, hi = std::min(nn, lo + ochunk);
            for (int k = 0; k < ha.n && e == cudaSuccess; ++k)
                e = cudaMemcpyAsync(static_cast<char *>(ha.a[k]) + lo * ha.es[k],
                                    static_cast<const char *>(hs.a[k]) + lo * ha.es[k], (hi - lo) * ha.es[k],
                                    cudaMemcpyDeviceToHost, down);
            if (e == cudaSuccess) e = cudaEventRecord(ev[c], down);
        }
        if (bytes) bytes[1] += nn * (int64_t)(ha.n == 7 ? 28 : 44) + (host_f ? 6 * (int64_t)fbytes : 0);
        prev_chunks = och;
        prev_chunk = ochunk;
        n = nn;
    }
    // `stream` completes after the last copies out
    cudaError_t e2 = cudaEventRecord(ev_end, down);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev_end, 0);
    if (e == cudaSuccess) e = e2;
    host->n = n;
    if (st) return st;
    return e == cudaSuccess ? GRPIC_OK : cuda_fail(ctx, e, "grpic_step_host");
}

grpic_status grpic_diagnostics(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, void *rho, void *divD,
                               void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f) || !divD || (rho && !particles_ok(ctx, p)))
        return fail(ctx, GRPIC_EINVAL, "grpic_diagnostics: bad arguments");
    cudaError_t e = launch_diag(ctx, rho ? p : nullptr, f, rho, divD, S(stream));
    return e == cudaSuccess ? GRPIC_OK : cuda_fail(ctx, e, "diagnostics");
}

grpic_status grpic_charge_check(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, const double *base,
                                double *state, double out[2], void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f) || !out || (p && !particles_ok(ctx, p)))
        return fail(ctx, GRPIC_EINVAL, "grpic_charge_check: bad arguments");
    const size_t n = (size_t)(ctx->g.nth + 1) * f->ld;
    double *rho = nullptr, *divD = nullptr;
    unsigned long long *dout = nullptr;
    cudaError_t e = cudaMalloc(&rho, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&divD, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = launch_charge_check(ctx, p, f, rho, divD, base, state, dout, S(stream));
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, S(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
    cudaFree(rho);
    cudaFree(divD);
    cudaFree(dout);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "charge check");
    memcpy(&out[0], &h[0], sizeof(double));
    memcpy(&out[1], &h[1], sizeof(double));
    return GRPIC_OK;
}

grpic_status grpic_get_areas(grpic_ctx *ctx, double *const out[6], int64_t ld, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!out || ld < ctx->g.ld_tab) return fail(ctx, GRPIC_EINVAL, "grpic_get_areas: bad arguments");
    const int slots[6] = {T_ADR, T_ADT, T_ADP, T_ABR, T_ABT, T_ABP};
    for (int k = 0; k < 6; ++k) {
        if (!out[k]) return fail(ctx, GRPIC_EINVAL, "grpic_get_areas: null output");
        cudaError_t e = cudaMemcpy2DAsync(out[k], ld * sizeof(double), ctx->tab + slots[k] * ctx->slab,
                                          ctx->g.ld_tab * sizeof(double), ctx->g.ld_tab * sizeof(double),
                                          ctx->g.nth + 1, cudaMemcpyDeviceToDevice, S(stream));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "get_areas");
    }
    return GRPIC_OK;
}

grpic_status grpic_sync(grpic_ctx *ctx, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    cudaError_t e = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    int st = 0;
    e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync status read");
    if (st) {
        cudaMemset(ctx->d_status, 0, sizeof(int));
        const char *what = st == GRPIC_ERANGE ? "a particle moved more than one cell"
                           : st == GRPIC_ENAN ? "a particle state became non-finite"
                           : st == GRPIC_ETIMEOUT ? "a device-side wait timed out"
                                                  : "device error";
        snprintf(ctx->err, sizeof ctx->err, "%s", what);
    }
    return (grpic_status)st;
}

const char *grpic_last_error(const grpic_ctx *ctx) { return ctx ? ctx->err : "null context"; }

grpic_status grpic_set_timing(grpic_ctx *ctx, int enable)
{
    if (!ctx) return GRPIC_EINVAL;
    ctx->timing = enable ? 1 : 0;
    ctx->tsteps = 0;
    return GRPIC_OK;
}

grpic_status grpic_get_timing(grpic_ctx *ctx, double out[3], int64_t *nsteps)
{
    if (!ctx || !out || !nsteps) return GRPIC_EINVAL;
    out[0] = out[1] = out[2] = 0.0;
    *nsteps = ctx->tsteps;
    for (int64_t k = 0; k < ctx->tsteps; ++k) {
        cudaEvent_t *ev = &(*ctx->tevents)[4 * (size_t)k];
        if (cudaEventSynchronize(ev[3]) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "timing");
        for (int ph = 0; ph < 3; ++ph) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "timing");
            out[ph] += ms;
        }
    }
    ctx->tsteps = 0;
    return GRPIC_OK;
}

// ---------------------------------------------------------------------------
// theta-slab decomposition: row-restricted field update, halos, migration
// ---------------------------------------------------------------------------
grpic_status grpic_field_update_rows(grpic_ctx *ctx, grpic_fields *f, int32_t j_lo, int32_t j_hi, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f) || j_lo < 0 || j_hi > ctx->g.nth + 1 || j_lo >= j_hi)
        return fail(ctx, GRPIC_EINVAL, "grpic_field_update_rows: bad arguments");
    grpic_status st = ensure_field_scratch(ctx, f->ld);
    if (st) return st;
    cudaError_t e = (ctx->prm.precision == 64) ? launch_field64(ctx, f, S(stream), j_lo, j_hi)
                                                : launch_field32(ctx, f, S(stream), j_lo, j_hi);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "field update (rows)");
    return GRPIC_OK;
}

grpic_status grpic_halo_pack(grpic_ctx *ctx, const grpic_fields *f, int32_t set, int32_t row0, int32_t nrows, void *buf,
                             void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f) || (set != 0 && set != 1) || row0 < 0 || nrows < 0 || row0 + nrows > ctx->g.nth + 1 ||
        (nrows > 0 && !buf))
        return fail(ctx, GRPIC_EINVAL, "grpic_halo_pack: bad arguments");
    const size_t n = (size_t)nrows * f->ld, off = (size_t)row0 * f->ld, es = fsize(ctx);
    void *comp[6] = {f->D[0], f->D[1], f->D[2], f->B[0], f->B[1], f->B[2]};
    void *jc[3] = {f->J[0], f->J[1], f->J[2]};
    const int nc = set == 0 ? 6 : 3;
    for (int k = 0; k < nc && n > 0; ++k) {
        const char *src = (const char *)(set == 0 ? comp[k] : jc[k]) + off * es;
        cudaError_t e = cudaMemcpyAsync((char *)buf + k * n * es, src, n * es, cudaMemcpyDeviceToDevice, S(stream));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "halo pack");
    }
    return GRPIC_OK;
}

grpic_status grpic_halo_unpack(grpic_ctx *ctx, grpic_fields *f, int32_t set, int32_t row0, int32_t nrows,
                               const void *buf, int32_t add, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!fields_ok(ctx, f) || (set != 0 && set != 1) || row0 < 0 || nrows < 0 || row0 + nrows > ctx->g.nth + 1 ||
        (nrows > 0 && !buf))
        return fail(ctx, GRPIC_EINVAL, "grpic_halo_unpack: bad arguments");
    const size_t n = (size_t)nrows * f->ld, off = (size_t)row0 * f->ld, es = fsize(ctx);
    void *comp[6] = {f->D[0], f->D[1], f->D[2], f->B[0], f->B[1], f->B[2]};
    void *jc[3] = {f->J[0], f->J[1], f->J[2]};
    const int nc = set == 0 ? 6 : 3;
    if (n == 0) return GRPIC_OK;
    if (!add) {
        for (int k = 0; k < nc; ++k) {
            char *dst = (char *)(set == 0 ? comp[k] : jc[k]) + off * es;
            cudaError_t e =
                cudaMemcpyAsync(dst, (const char *)buf + k * n * es, n * es, cudaMemcpyDeviceToDevice, S(stream));
            if (e != cudaSuccess) return cuda_fail(ctx, e, "halo unpack");
        }
        return GRPIC_OK;
    }
    const size_t total = (size_t)nc * n;
    const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 4096);
    if (ctx->prm.precision == 64) {
        HaloComps<double> P;
        for (int k = 0; k < 6; ++k) P.p[k] = k < nc ? (double *)(set == 0 ? comp[k] : jc[k]) : nullptr;
        halo_add_kernel<double><<<blocks, 256, 0, S(stream)>>>(P, nc, off, n, (const double *)buf);
    } else {
        HaloComps<float> P;
        for (int k = 0; k < 6; ++k) P.p[k] = k < nc ? (float *)(set == 0 ? comp[k] : jc[k]) : nullptr;
        halo_add_kernel<float><<<blocks, 256, 0, S(stream)>>>(P, nc, off, n, (const float *)buf);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "halo add");
    return GRPIC_OK;
}

grpic_status grpic_sort_split(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, int32_t j_lo,
                              int32_t j_hi, int64_t counts[3], void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!particles_ok(ctx, p) || !particles_ok(ctx, scratch) || scratch->capacity < p->n || !counts || j_lo < 0 ||
        j_hi > ctx->g.nth || j_lo > j_hi || ctx->pending_perm)
        return fail(ctx, GRPIC_EINVAL, "grpic_sort_split: bad arguments");
    drop_sort_state(ctx);  // keys recomputed from the positions, general counting sort
    grpic_status st = sort_impl(ctx, p, scratch, S(stream));
    if (st) return st;
    // segment starts of the new order: rows below j_lo, rows [j_lo, j_hi), the rest live
    const int64_t nr = ctx->g.nr, ncell = nr * ctx->g.nth;
    int32_t o[3] = {0, 0, 0};
    cudaStream_t s = S(stream);
    cudaError_t e = cudaMemcpyAsync(&o[0], ctx->d_offset_prev + (int64_t)j_lo * nr, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&o[1], ctx->d_offset_prev + (int64_t)j_hi * nr, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&o[2], ctx->d_offset_prev + ncell, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sort split");
    counts[0] = o[0];
    counts[1] = o[1] - o[0];
    counts[2] = o[2] - o[1];
    return GRPIC_OK;
}

grpic_status grpic_particles_pack(grpic_ctx *ctx, const grpic_particles *p, int64_t first, int64_t n, void *buf,
                                  void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    if (!p || first < 0 || n < 0 || first + n > p->capacity || (n > 0 && !buf) ||
        (n > 0 && !particles_ok(ctx, p)))
        return fail(ctx, GRPIC_EINVAL, "grpic_particles_pack: bad arguments");
    void *arr[7];
    size_t esz[7];
    const int na = particle_arrays(ctx, p, arr, esz);
    size_t off = 0;
    for (int k = 0; k < na && n > 0; ++k) {
        cudaError_t e = cudaMemcpyAsync((char *)buf + off, (const char *)arr[k] + first * esz[k], n * esz[k],
                                        cudaMemcpyDeviceToDevice, S(stream));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "particles pack");
        off += n * esz[k];
    }
    return GRPIC_OK;
}

grpic_status grpic_slab_assemble(grpic_ctx *ctx, grpic_particles *dst, const grpic_particles *src, int64_t own_first,
                                 int64_t own_n, const void *lower, int64_t n_lower, const void *upper,
                                 int64_t n_upper, void *stream)
{
    if (!ctx) return GRPIC_EINVAL;
    const int64_t total = n_lower + own_n + n_upper;
    if (!dst || !src || own_first < 0 || own_n < 0 || n_lower < 0 || n_upper < 0 || own_first + own_n > src->capacity ||
        total > dst->capacity || total > INT32_MAX || (n_lower > 0 && !lower) || (n_upper > 0 && !upper) ||
        !dst->x1 || !dst->x2 || !dst->u1 || !dst->u2 || !dst->u3 || !dst->tag ||
        (ctx->prm.precision == 32 && !dst->cell) || (own_n > 0 && !particles_ok(ctx, src)))
        return fail(ctx, GRPIC_EINVAL, "grpic_slab_assemble: bad arguments");
    cudaStream_t s = S(stream);
    void *da[7], *sa[7];
    size_t esz[7];
    const int na = particle_arrays(ctx, dst, da, esz);
    particle_arrays(ctx, src, sa, esz);
    size_t ol = 0, ou = 0;
    for (int k = 0; k < na; ++k) {
        char *d = (char *)da[k];
        cudaError_t e = cudaSuccess;
        if (n_lower > 0) e = cudaMemcpyAsync(d, (const char *)lower + ol, n_lower * esz[k], cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && own_n > 0)
            e = cudaMemcpyAsync(d + n_lower * esz[k], (const char *)sa[k] + own_first * esz[k], own_n * esz[k],
                                cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && n_upper > 0)
            e = cudaMemcpyAsync(d + (n_lower + own_n) * esz[k], (const char *)upper + ou, n_upper * esz[k],
                                cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "slab assemble");
        ol += n_lower * esz[k];
        ou += n_upper * esz[k];
    }
    dst->n = total;
    if (dst->d_count) {
        cudaError_t e = cudaMemcpyAsync(dst->d_count, &dst->n, sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host source lives in the caller's struct
        if (e != cudaSuccess) return cuda_fail(ctx, e, "slab assemble count");
    }
    drop_sort_state(ctx);
    return GRPIC_OK;
}

grpic_status grpic_set_field_path(grpic_ctx *ctx, int32_t fused)
{
    if (!ctx) return GRPIC_EINVAL;
    ctx->field_fused = fused ? 1 : 0;
    return GRPIC_OK;
}

void grpic_destroy(grpic_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->tevents) {
        for (cudaEvent_t e : *ctx->tevents) cudaEventDestroy(e);
        delete ctx->tevents;
    }
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->hevents) {
        for (cudaEvent_t e : *ctx->hevents) cudaEventDestroy(e);
        delete ctx->hevents;
    }
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->down_stream) cudaStreamDestroy(ctx->down_stream);
    if (ctx->h_count) cudaFreeHost(ctx->h_count);
    void *ptrs[] = {ctx->d_spawn, ctx->d_rad, ctx->d_spqm, ctx->d_spmassive, ctx->d_offset_prev, ctx->d_cnt9, ctx->d_base9, ctx->d_sortflag, ctx->rcol, ctx->rcol2, ctx->rowsc, ctx->tab, ctx->col1d, ctx->tab32, ctx->col1d32, ctx->fscratch, ctx->q32, ctx->d_status, ctx->d_keys,
                    ctx->d_count, ctx->d_offset, ctx->d_cursor, ctx->d_blocksum, ctx->d_perm, ctx->d_bigseg};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete ctx;
}

}  // extern "C"
