// grpic_adjoint_spin.cu -- the full spin derivative of the differentiable
// form's objective for a run that starts from an analytic field (App. C).
//
// L depends on the spin a through the metric of every push and field update
// at fixed step-0 state (the part grpic_adjoint_grad returns) and through
// the step-0 fields themselves when they are the closed-form solution of that
// spin: dL/da = (dL/da at fixed F0) + sum over every entry of
// dL/dF0 . dF0/da.  dF0/da is the central difference (h = 1e-5) of the
// closed-form initialization at a +- h, each with the face areas of its own
// spin (Stokes' theorem divides the potential differences by the areas): the
// same treatment the adjoint gives the tables, smooth in a, truncation ~h^2.
// The horizon index of the objective (the column nearest the outer horizon)
// is also computed here.
#include "grpic_internal.cuh"

#include <cmath>
#include <vector>

namespace grpic {
namespace {

constexpr int RED_THREADS = 256;

// out += sum_k sum_q g_k[q] (p_k[q] - m_k[q]) * scale over the six arrays
__global__ void __launch_bounds__(RED_THREADS) contract_kernel(const double *const *g, const double *const *p,
                                                               const double *const *m, size_t n, double scale,
                                                               double *out)
{
    __shared__ double part[RED_THREADS / 32];
    double acc = 0.0;
    for (int k = 0; k < 6; ++k) {
        const double *gk = g[k], *pk = p[k], *mk = m[k];
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
            acc += gk[q] * (pk[q] - mk[q]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < RED_THREADS / 32 ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc * scale);
    }
}

}  // namespace
}  // namespace grpic

using namespace grpic;

extern "C" grpic_status grpic_horizon_index(const grpic_ctx *ctx, double a_nominal, int32_t *out)
{
    if (!ctx || !out || !(a_nominal >= 0.0 && a_nominal < 1.0)) return GRPIC_EINVAL;
    const double rh = 1.0 + std::sqrt(1.0 - a_nominal * a_nominal);
    const double x = std::log(rh / ctx->g.r_in) / ctx->g.dx1;
    *out = (int32_t)std::lround(x);
    return GRPIC_OK;
}

extern "C" grpic_status grpic_adjoint_spin(grpic_ctx *ctx, const grpic_particles *p0, grpic_field_kind kind,
                                           double B0, int nsteps, int checkpoint_every, int i_horizon,
                                           int trapezoid_ift, double *L_out, double *const grad_p[5],
                                           double *const grad_f[6], double *dL_da, void *stream)
{
    if (!ctx || !p0 || !L_out || !grad_p || !dL_da || ctx->prm.precision != 64 || (int)kind < 0 || (int)kind > 3)
        return GRPIC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ld = ctx->g.ld_tab;
    const size_t fn = (size_t)(ctx->g.nth + 1) * ld;
    std::vector<void *> allocs;
    auto dalloc = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
        allocs.push_back(q);
        return q;
    };
    auto release = [&](grpic_status st) {
        for (void *q : allocs) cudaFree(q);
        return st;
    };
    // step-0 fields at the context's spin, fields at a +- h, the two table
    // sets, the gradient w.r.t. F0 when the caller does not keep it
    double *F0 = (double *)dalloc(9 * fn * sizeof(double));
    double *Fp = (double *)dalloc(9 * fn * sizeof(double));
    double *Fm = (double *)dalloc(9 * fn * sizeof(double));
    double *tp = (double *)dalloc((size_t)T_COUNT * ctx->slab * sizeof(double));
    double *tm = (double *)dalloc((size_t)T_COUNT * ctx->slab * sizeof(double));
    double *c1 = (double *)dalloc(4 * (size_t)ld * sizeof(double));
    bool own_gf = false;
    for (int k = 0; k < 6; ++k) own_gf = own_gf || !grad_f || !grad_f[k];
    double *gfo = own_gf ? (double *)dalloc(6 * fn * sizeof(double)) : nullptr;
    double **dptr = (double **)dalloc(18 * sizeof(double *));
    double *acc = (double *)dalloc(sizeof(double));
    if (!F0 || !Fp || !Fm || !tp || !tm || !c1 || (own_gf && !gfo) || !dptr || !acc) return release(GRPIC_ENOMEM);
    auto fields_of = [&](double *base) {
        grpic_fields f;
        for (int k = 0; k < 3; ++k) {
            f.D[k] = base + k * fn;
            f.B[k] = base + (3 + k) * fn;
            f.J[k] = base + (6 + k) * fn;
        }
        f.ld = ld;
        return f;
    };
    grpic_fields f0 = fields_of(F0), fp = fields_of(Fp), fm = fields_of(Fm);
    if (launch_init_fields(ctx, (int)kind, B0, &f0, s) != cudaSuccess) return release(GRPIC_ECUDA);
    double *gf[6];
    for (int k = 0; k < 6; ++k) gf[k] = own_gf ? gfo + k * fn : grad_f[k];
    double La = 0.0;
    grpic_status st = grpic_adjoint_grad(ctx, p0, &f0, nsteps, checkpoint_every, i_horizon, trapezoid_ift, L_out,
                                         grad_p, gf, &La, stream);
    if (st != GRPIC_OK && st != GRPIC_ERANGE && st != GRPIC_ENAN) return release(st);
    // dF0/da: the closed forms at a +- h with the areas of a +- h
    const double h = 1e-5;
    if (launch_tables_at(ctx, ctx->g.a + h, tp, c1, s) != cudaSuccess ||
        launch_tables_at(ctx, ctx->g.a - h, tm, c1, s) != cudaSuccess ||
        launch_init_fields_at(ctx, ctx->g.a + h, tp, (int)kind, B0, &fp, s) != cudaSuccess ||
        launch_init_fields_at(ctx, ctx->g.a - h, tm, (int)kind, B0, &fm, s) != cudaSuccess)
        return release(GRPIC_ECUDA);
    const double *hp[18];
    for (int k = 0; k < 6; ++k) {
        hp[k] = gf[k];
        hp[6 + k] = Fp + k * fn;   // D^r .. D^phi then B^r .. B^phi: the first six arrays of a field set
        hp[12 + k] = Fm + k * fn;
    }
    if (cudaMemcpyAsync(dptr, hp, sizeof hp, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(acc, 0, sizeof(double), s) != cudaSuccess)
        return release(GRPIC_ECUDA);
    int nsm = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    contract_kernel<<<2 * nsm, RED_THREADS, 0, s>>>(dptr, dptr + 6, dptr + 12, fn, 1.0 / (2.0 * h), acc);
    double dF = 0.0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&dF, acc, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return release(GRPIC_ECUDA);
    *dL_da = La + dF;
    return release(st);
}
