// grpic_rad.cu -- 2D photon emission, pair conversion (the prescription of
// Sec. 4 on the 2D grid) and the pair injection of the plasma-filled Wald
// run (Sec. 3.4), FP64 path.
//
// The push decides per slot (see push64_kernel): a charged particle whose
// FIDO Lorentz factor Gamma = sqrt(1 + gamma^ij u_i u_j) reaches gamma_thr
// emits a photon of FIDO energy eps_ph along its momentum and keeps the
// rest (spawn 1); a photon of FIDO energy e > 2 converts with probability
// 1 - exp(-tau dt) (uniform from Philox keyed on the slot and the step;
// spawn 2) and dies.  Here the children are appended after all slots in
// parent order: per block of 1024 slots the spawn counts are summed, the
// sums scanned, and each block places its children in slot order (a
// photon with k_i = eps_ph u_i / |u| at its emitter; an e- then an e+ with
// u = s k, s = sqrt((e/2)^2 - 1)/e, at the photon).  The order is the same
// as a serial pass, so a stable sort afterwards is deterministic.
//
// Injection, after the field update: per cell (c = j n_r + i), with the
// fields interpolated to the cell centre (i + 1/2, j + 1/2) by the shape in
// use, B^2 = gamma_ij B^i B^j, D.B = gamma_ij D^i B^j, and the density
// n = max(1, charged live particles in the cell) |q w_0| / V_cell (V_cell =
// A^B_phi): where B^2 / n > sigma_thr and |D.B| / B^2 > eps_db an e- and an
// e+ start at rest in the FIDO frame (u_i = 0) at (i + U1, j + U2), U1, U2
// from Philox keyed on the cell and the step (events 2, 3); appended in cell
// order after the children.
#include "grpic_internal.cuh"
#include "grpic_philox.cuh"
#include "grpic_shape3.cuh"

namespace grpic {
namespace {

constexpr int RB = 1024;  // slots (or cells) per block of the ordered appends
constexpr int RT = 256;   // threads per block: four slots each

__device__ __forceinline__ int jcl(const GridDev &g, double x2)
{
    int j = (int)floor(x2);
    return j > g.nth - 1 ? g.nth - 1 : j;
}

__device__ __forceinline__ int key_of(const GridDev &g, double r, double th)
{
    int i = (int)floor((log(r) - g.ln_rin) / g.dx1);
    i = i < 0 ? 0 : (i > g.nr - 1 ? g.nr - 1 : i);
    return jcl(g, th / g.dth) * g.nr + i;
}

// block-exclusive scan of 4 values per thread (slot order = thread-major
// quadruples); returns the block total
__device__ int block_scan4(int v[4], int *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int t = v[0] + v[1] + v[2] + v[3];
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < RT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < RT / 32) sh[lane] = x;  // inclusive warp totals
    }
    __syncthreads();
    int base = (w > 0 ? sh[w - 1] : 0) + incl - t;
    const int total = sh[RT / 32 - 1];
    __syncthreads();
    int run = base;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = v[k];
        v[k] = run;
        run += x;
    }
    return total;
}

// per block of RB entries: the sum of per-entry counts (spawn counts of the
// slots [0, *n) or flags of the cells [0, n))
__global__ void __launch_bounds__(RT) block_sums(const int32_t *cnt, const int64_t *d_n, int64_t n_fixed,
                                                 int64_t nmax, int32_t *bsum)
{
    __shared__ int sh[RT / 32];
    int64_t n = d_n ? *d_n : n_fixed;
    if (n > nmax) n = nmax;
    const int64_t base = (int64_t)blockIdx.x * RB + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = base + k < n ? cnt[base + k] : 0;
    const int total = block_scan4(v, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

struct AppendArgs {
    GridDev g;
    int64_t nmax, cap;
    int64_t *d_count;
    const int32_t *spawn, *boff;
    double *r, *th, *u1, *u2, *u3;
    uint32_t *tag;
    int32_t *keys;
    double eps_ph;
    int *status;
};

// children of the slots of this block at *d_count + boff[b] + (rank in slot order)
__global__ void __launch_bounds__(RT) append_children(AppendArgs A)
{
    __shared__ int sh[RT / 32];
    int64_t n = *A.d_count;
    if (n > A.nmax) n = A.nmax;
    const int64_t base = (int64_t)blockIdx.x * RB + 4 * threadIdx.x;
    int v[4], sp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = sp[k] = base + k < n ? A.spawn[base + k] : 0;
    block_scan4(v, sh);
    const int64_t at0 = n + A.boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (sp[k] == 0) continue;
        const int64_t p = base + k;
        const double r = A.r[p], th = A.th[p];
        const double k1 = A.u1[p], k2 = A.u2[p], k3 = A.u3[p];
        KS m;
        ks_point(A.g.a, r, th, m);
        const double uu = m.gi_rr * k1 * k1 + 2.0 * m.gi_rp * k1 * k3 + m.gi_tt * k2 * k2 + m.gi_pp * k3 * k3;
        const int key = key_of(A.g, r, th);
        int64_t at = at0 + v[k];
        if (sp[k] == 1) {
            // the photon along the (reduced) momentum of its emitter
            const double f = A.eps_ph / sqrt(uu);
            if (at >= A.cap) {
                set_status(A.status, GRPIC_EOVERFLOW);
                continue;
            }
            A.r[at] = r;
            A.th[at] = th;
            A.u1[at] = f * k1;
            A.u2[at] = f * k2;
            A.u3[at] = f * k3;
            A.tag[at] = 3u;
            A.keys[at] = key;
        } else {
            const double e = sqrt(uu), s = sqrt(0.25 * e * e - 1.0) / e;
            for (int c = 0; c < 2; ++c, ++at) {
                if (at >= A.cap) {
                    set_status(A.status, GRPIC_EOVERFLOW);
                    break;
                }
                A.r[at] = r;
                A.th[at] = th;
                A.u1[at] = s * k1;
                A.u2[at] = s * k2;
                A.u3[at] = s * k3;
                A.tag[at] = (uint32_t)c;
                A.keys[at] = key;
            }
        }
    }
}

// *d_count += per * total (clamped to the capacity)
__global__ void count_add(int64_t *d_count, const int32_t *total, int per, int64_t cap)
{
    int64_t v = *d_count + (int64_t)per * (*total);
    *d_count = v > cap ? cap : v;
}

// charged live particles per cell
__global__ void charged_per_cell(GridDev g, const int64_t *d_count, int64_t nmax, const double *r, const double *th,
                                 const uint32_t *tag, const double *qm, const int *massive, int32_t *nq)
{
    int64_t n = *d_count;
    if (n > nmax) n = nmax;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t t = tag[p];
    if (t & DEAD) return;
    const int sp = t & 3u;
    if (!(massive[sp] && qm[sp] != 0.0)) return;
    const double x1 = (log(r[p]) - g.ln_rin) / g.dx1;
    const int i = (int)floor(x1), j = jcl(g, th[p] / g.dth);
    if (i < 0 || i >= g.nr || j < 0) return;
    atomicAdd(nq + (size_t)j * g.nr + i, 1);
}

// bilinear field at logical (x1, x2) on a lattice staggered by sr (half rows
// if half_t; par = parity across the axis)
__device__ double cic_at(const double *F, int64_t ld, int nth, double x1, double x2, double sr, bool half_t,
                         double par)
{
    const double xi = x1 - sr, eta = x2 - (half_t ? 0.5 : 0.0);
    int i = (int)floor(xi), j = (int)floor(eta);
    if (!half_t && j > nth - 1) j = nth - 1;
    const double f = xi - i, h = eta - j;
    double v = 0.0;
    for (int b = 0; b < 2; ++b) {
        bool flip;
        const int jj = mirror_row(j + b, half_t, nth, flip);
        const double *row = F + (size_t)jj * ld + (i + NG);
        const double w = (b ? h : 1.0 - h) * (flip ? par : 1.0);
        v += w * ((1.0 - f) * row[0] + f * row[1]);
    }
    return v;
}

struct InjArgs {
    GridDev g;
    const double *D0, *D1, *D2, *B0, *B1, *B2;
    int64_t ld;
    const double *tab;
    size_t slab;
    const int32_t *nq;
    double w0, sigma_thr, eps_db;
    int shape;
    int32_t *flag;
};

__global__ void inject_flags(InjArgs A)
{
    const int64_t ncell = (int64_t)A.g.nr * A.g.nth;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int i = (int)(c % A.g.nr), j = (int)(c / A.g.nr);
    const double x1 = i + 0.5, x2 = j + 0.5;
    double Dv[3], Bv[3];
    if (A.shape == 3) {
        gather3_fields(A.D0, A.D1, A.D2, A.B0, A.B1, A.B2, A.ld, A.g.nth, x1, x2, Dv, Bv);
    } else {
        Dv[0] = cic_at(A.D0, A.ld, A.g.nth, x1, x2, 0.5, false, 1.0);
        Dv[1] = cic_at(A.D1, A.ld, A.g.nth, x1, x2, 0.0, true, -1.0);
        Dv[2] = cic_at(A.D2, A.ld, A.g.nth, x1, x2, 0.0, false, 1.0);
        Bv[0] = cic_at(A.B0, A.ld, A.g.nth, x1, x2, 0.0, true, 1.0);
        Bv[1] = cic_at(A.B1, A.ld, A.g.nth, x1, x2, 0.5, false, 1.0);
        Bv[2] = cic_at(A.B2, A.ld, A.g.nth, x1, x2, 0.5, true, 1.0);
    }
    KS m;
    ks_point(A.g.a, A.g.r_in * exp(x1 * A.g.dx1), x2 * A.g.dth, m);
    const double Bl0 = m.g_rr * Bv[0] + m.g_rp * Bv[2], Bl1 = m.g_tt * Bv[1], Bl2 = m.g_rp * Bv[0] + m.g_pp * Bv[2];
    const double B2 = Bl0 * Bv[0] + Bl1 * Bv[1] + Bl2 * Bv[2];
    const double DB = Bl0 * Dv[0] + Bl1 * Dv[1] + Bl2 * Dv[2];
    const double V = A.tab[T_ABP * A.slab + (size_t)j * A.g.ld_tab + (i + NG)];
    const int q = A.nq[c];
    const double n = (q > 0 ? (double)q : 1.0) * A.w0 / V;
    A.flag[c] = (B2 > 0.0 && B2 / n > A.sigma_thr && fabs(DB) / B2 > A.eps_db) ? 1 : 0;
}

struct PairArgs {
    GridDev g;
    int64_t cap;
    int64_t *d_count;
    const int32_t *flag, *boff;
    double *r, *th, *u1, *u2, *u3;
    uint32_t *tag;
    int32_t *keys;
    uint64_t seed;
    int64_t step;
    int *status;
};

__global__ void __launch_bounds__(RT) append_pairs(PairArgs A)
{
    __shared__ int sh[RT / 32];
    const int64_t ncell = (int64_t)A.g.nr * A.g.nth;
    const int64_t n = *A.d_count;
    const int64_t base = (int64_t)blockIdx.x * RB + 4 * threadIdx.x;
    int v[4], fl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = fl[k] = base + k < ncell ? A.flag[base + k] : 0;
    block_scan4(v, sh);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!fl[k]) continue;
        const int64_t c = base + k;
        const int i = (int)(c % A.g.nr), j = (int)(c / A.g.nr);
        const double U1 = uniform53(A.seed, (uint64_t)c, A.step, 2), U2 = uniform53(A.seed, (uint64_t)c, A.step, 3);
        const double rr = A.g.r_in * exp((i + U1) * A.g.dx1), tt = (j + U2) * A.g.dth;
        int64_t at = n + 2 * ((int64_t)A.boff[blockIdx.x] + v[k]);
        for (int s = 0; s < 2; ++s, ++at) {
            if (at >= A.cap) {
                set_status(A.status, GRPIC_EOVERFLOW);
                break;
            }
            A.r[at] = rr;
            A.th[at] = tt;
            A.u1[at] = 0.0;
            A.u2[at] = 0.0;
            A.u3[at] = 0.0;
            A.tag[at] = (uint32_t)s;
            A.keys[at] = (int32_t)c;
        }
    }
}

}  // namespace

cudaError_t ensure_rad_scratch(grpic_ctx *ctx, int64_t cap)
{
    const int64_t ncell = (int64_t)ctx->g.nr * ctx->g.nth;
    if (ctx->rad_cap >= cap && ctx->d_spawn) return cudaSuccess;
    cudaFree(ctx->d_spawn);
    cudaFree(ctx->d_rad);
    ctx->d_spawn = nullptr;
    ctx->d_rad = nullptr;
    const int64_t nbp = (cap + RB - 1) / RB, nbc = (ncell + RB - 1) / RB;
    cudaError_t e = cudaMalloc(&ctx->d_spawn, sizeof(int32_t) * (size_t)cap);
    // rad: [block sums / offsets of slots: nbp + 1] [of cells: nbc + 1] [charged per cell: ncell] [flags: ncell]
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->d_rad, sizeof(int32_t) * (size_t)(2 * (nbp + 1) + 2 * (nbc + 1) + 2 * ncell));
    ctx->rad_cap = e == cudaSuccess ? cap : 0;
    return e;
}

// the children of the last push's spawn decisions, after the live slots
cudaError_t launch_append_children(grpic_ctx *ctx, grpic_particles *p, cudaStream_t s)
{
    const int64_t nbp = (p->capacity + RB - 1) / RB;
    int32_t *bsum = ctx->d_rad, *boff = bsum + (nbp + 1);
    block_sums<<<(unsigned)nbp, RT, 0, s>>>(ctx->d_spawn, p->d_count, p->n, p->capacity, bsum);
    cudaError_t e = launch_scan_i32(bsum, boff, ctx->d_blocksum, nbp, s);
    if (e != cudaSuccess) return e;
    AppendArgs A;
    A.g = ctx->g;
    A.nmax = p->capacity;
    A.cap = p->capacity;
    A.d_count = p->d_count;
    A.spawn = ctx->d_spawn;
    A.boff = boff;
    A.r = (double *)p->x1;
    A.th = (double *)p->x2;
    A.u1 = (double *)p->u1;
    A.u2 = (double *)p->u2;
    A.u3 = (double *)p->u3;
    A.tag = p->tag;
    A.keys = ctx->d_keys;
    A.eps_ph = ctx->prm.eps_ph;
    A.status = ctx->d_status;
    append_children<<<(unsigned)nbp, RT, 0, s>>>(A);
    count_add<<<1, 1, 0, s>>>(p->d_count, boff + nbp, 1, p->capacity);
    return cudaGetLastError();
}

// pair injection after the field update
cudaError_t launch_injection(grpic_ctx *ctx, grpic_particles *p, const grpic_fields *f, cudaStream_t s)
{
    const int64_t ncell = (int64_t)ctx->g.nr * ctx->g.nth;
    const int64_t nbp = (p->capacity + RB - 1) / RB, nbc = (ncell + RB - 1) / RB;
    int32_t *cbsum = ctx->d_rad + 2 * (nbp + 1), *cboff = cbsum + (nbc + 1);
    int32_t *nq = cboff + (nbc + 1), *flag = nq + ncell;
    cudaMemsetAsync(nq, 0, sizeof(int32_t) * (size_t)ncell, s);
    const unsigned gp = (unsigned)((p->capacity + 255) / 256);
    charged_per_cell<<<gp, 256, 0, s>>>(ctx->g, p->d_count, p->capacity, (const double *)p->x1,
                                        (const double *)p->x2, p->tag, ctx->d_spqm, ctx->d_spmassive, nq);
    InjArgs I;
    I.g = ctx->g;
    I.D0 = (const double *)f->D[0];
    I.D1 = (const double *)f->D[1];
    I.D2 = (const double *)f->D[2];
    I.B0 = (const double *)f->B[0];
    I.B1 = (const double *)f->B[1];
    I.B2 = (const double *)f->B[2];
    I.ld = f->ld;
    I.tab = ctx->tab;
    I.slab = ctx->slab;
    I.nq = nq;
    I.w0 = fabs(ctx->prm.q_weight[0]);
    I.sigma_thr = ctx->prm.sigma_thr;
    I.eps_db = ctx->prm.eps_db;
    I.shape = ctx->prm.shape_order;
    I.flag = flag;
    inject_flags<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(I);
    block_sums<<<(unsigned)nbc, RT, 0, s>>>(flag, nullptr, ncell, ncell, cbsum);
    cudaError_t e = launch_scan_i32(cbsum, cboff, ctx->d_blocksum, nbc, s);
    if (e != cudaSuccess) return e;
    PairArgs P;
    P.g = ctx->g;
    P.cap = p->capacity;
    P.d_count = p->d_count;
    P.flag = flag;
    P.boff = cboff;
    P.r = (double *)p->x1;
    P.th = (double *)p->x2;
    P.u1 = (double *)p->u1;
    P.u2 = (double *)p->u2;
    P.u3 = (double *)p->u3;
    P.tag = p->tag;
    P.keys = ctx->d_keys;
    P.seed = ctx->prm.seed;
    P.step = ctx->step_count;
    P.status = ctx->d_status;
    append_pairs<<<(unsigned)nbc, RT, 0, s>>>(P);
    count_add<<<1, 1, 0, s>>>(p->d_count, cboff + nbc, 2, p->capacity);
    return cudaGetLastError();
}

}  // namespace grpic
