// grpic_sort.cu -- stable counting sort of the particles by cell key
// (key = j*n_r + i, dead = n_cells), which keeps the deposit's memory accesses
// coherent.  Not part of the paper's method; the order it produces is the one
// of a stable sort (equal keys keep their input order), so it is deterministic.
//
//   1. histogram of the keys (fused into the push, or the keys kernel here);
//   2. exclusive scan of the n_cells+1 counts: per-block scans with warp
//      shuffles, a scan of the block sums, an add-back pass;
//   3. scatter of slot indices: lanes of a warp holding the same key take
//      consecutive ranks from one atomicAdd on the key's cursor, so within a
//      key the indices arrive as runs in input order, runs in arbitrary order;
//   4. each key's segment of indices is sorted ascending (a warp per segment,
//      bitonic network in registers or shared memory; one block per segment
//      for segments beyond the warp's capacity) -- this restores input order,
//      i.e. stability;
//   5. gather of every particle array through the index list into the second
//      buffer; slots past the live count are marked dead.
#include "grpic_internal.cuh"

#include <climits>

namespace grpic {
namespace {

constexpr int SCAN_T = 1024, SCAN_IPT = 8, SCAN_TILE = SCAN_T * SCAN_IPT;
constexpr int SEG_WARP_MAX = 2048;  // largest segment sorted by one warp in smem
constexpr int SEG_BLOCK_MAX = 16384;
constexpr int SEG_WARPS = 4;

__device__ __forceinline__ int warp_incl_scan(int v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// block-wide exclusive scan of SCAN_IPT items per thread; returns block total
__device__ int block_scan(int (&v)[SCAN_IPT], int *sh)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int run = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        int t = v[k];
        v[k] = run;
        run += t;
    }
    int incl = warp_incl_scan(run);
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < SCAN_T / 32) ? sh[lane] : 0;
        int wi = warp_incl_scan(w);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    int base = sh[warp] + incl - run;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) v[k] += base;
    int total = sh[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_T) scan_tiles(const int32_t *in, int32_t *out, int32_t *bsum, int64_t n)
{
    __shared__ int sh[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    int v[SCAN_IPT];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) v[k] = (base + k < n) ? in[base + k] : 0;
    int total = block_scan(v, sh);
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k)
        if (base + k < n) out[base + k] = v[k];
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// single block: exclusive scan of the block sums (<= SCAN_TILE of them);
// writes the grand total to out_total
__global__ void __launch_bounds__(SCAN_T) scan_sums(int32_t *bsum, int nb, int32_t *out_total)
{
    __shared__ int sh[33];
    int base = threadIdx.x * SCAN_IPT;
    int v[SCAN_IPT];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) v[k] = (base + k < nb) ? bsum[base + k] : 0;
    int total = block_scan(v, sh);
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k)
        if (base + k < nb) bsum[base + k] = v[k];
    if (threadIdx.x == 0) *out_total = total;
}

__global__ void add_back(int32_t *out, const int32_t *bsum, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_TILE];
}

template <bool FP64>
__global__ void keys_kernel(GridDev g, int64_t nmax, const int64_t *d_count, const void *x1, const void *x2,
                            const int32_t *cell, const uint32_t *tag, int32_t *keys, int32_t *count)
{
    int64_t n = d_count ? *d_count : nmax;
    if (n > nmax) n = nmax;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ncell = g.nr * g.nth;
    int key = -1;
    if (p < n) {
        key = ncell;
        if (!(tag[p] & DEAD)) {
            if (FP64) {
                double r = ((const double *)x1)[p], th = ((const double *)x2)[p];
                int i = (int)floor((log(r) - g.ln_rin) / g.dx1);
                int j = (int)floor(th / g.dth);
                if (j > g.nth - 1) j = g.nth - 1;
                if (i >= 0 && i < g.nr && j >= 0) key = j * g.nr + i;
            } else {
                int c = cell[p];
                if (c >= 0 && c < ncell) key = c;
            }
        }
        keys[p] = key;
    }
    unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
}

__global__ void scatter_kernel(int64_t nmax, const int64_t *d_count, const int32_t *keys, const int32_t *offset,
                               int32_t *cursor, int32_t *perm, int ncell)
{
    int64_t n = d_count ? *d_count : nmax;
    if (n > nmax) n = nmax;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int key = (p < n) ? keys[p] : -1;
    if (key == ncell) key = -1;  // dead particles are dropped
    unsigned peers = __match_any_sync(0xffffffffu, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int base = 0;
    if (key >= 0 && lane == leader) base = atomicAdd(cursor + key, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (key >= 0) {
        int rank = __popc(peers & ((1u << lane) - 1u));
        perm[offset[key] + base + rank] = (int32_t)p;
    }
}

// compare-exchange network of the "flip" bitonic sort: only ascending
// exchanges, so values past the segment end behave as +infinity and their
// exchanges are no-ops.
__device__ __forceinline__ int warp_sort32(int v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
        int partner = lane ^ (k - 1);
        int o = __shfl_xor_sync(0xffffffffu, v, k - 1);
        v = (lane < partner) ? min(v, o) : max(v, o);
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            int o2 = __shfl_xor_sync(0xffffffffu, v, j);
            v = ((lane & j) == 0) ? min(v, o2) : max(v, o2);
        }
    }
    return v;
}

__device__ void smem_sort_warp(int *s, int m)
{
    int lane = threadIdx.x & 31;
    int N = 1;
    while (N < m) N <<= 1;
    for (int k = 2; k <= N; k <<= 1) {
        for (int i = lane; i < N; i += 32) {
            int l = i ^ (k - 1);
            if (l > i && l < m) {
                int a = s[i], b = s[l];
                if (b < a) { s[i] = b; s[l] = a; }
            }
        }
        __syncwarp();
        for (int j = k >> 2; j > 0; j >>= 1) {
            for (int i = lane; i < N; i += 32) {
                int l = i ^ j;
                if (l > i && l < m) {
                    int a = s[i], b = s[l];
                    if (b < a) { s[i] = b; s[l] = a; }
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(SEG_WARPS * 32) segfix_kernel(const int32_t *offset, int32_t *perm, int ncell,
                                                                 int32_t *bigseg, int32_t *nbig, int32_t *status)
{
    __shared__ int sh[SEG_WARPS][SEG_WARP_MAX];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t cellk = (int64_t)blockIdx.x * SEG_WARPS + warp;
    if (cellk >= ncell) return;
    int start = offset[cellk];
    int m = offset[cellk + 1] - start;
    if (m <= 1) return;
    int32_t *seg = perm + start;
    // already in order?  (the usual case for cells nobody entered)
    bool ok = true;
    for (int i = lane; i + 1 < m; i += 32) ok &= seg[i] <= seg[i + 1];
    if (__all_sync(0xffffffffu, ok)) return;
    if (m <= 32) {
        int v = lane < m ? seg[lane] : INT_MAX;
        v = warp_sort32(v);
        if (lane < m) seg[lane] = v;
    } else if (m <= SEG_WARP_MAX) {
        int *s = sh[warp];
        for (int i = lane; i < m; i += 32) s[i] = seg[i];
        __syncwarp();
        smem_sort_warp(s, m);
        for (int i = lane; i < m; i += 32) seg[i] = s[i];
    } else if (lane == 0) {
        int k = atomicAdd(nbig, 1);
        bigseg[k] = (int32_t)cellk;
    }
    (void)status;
}

// one block per oversized segment: bitonic network in shared memory when it
// fits, in global memory otherwise
__global__ void __launch_bounds__(1024) bigseg_kernel(const int32_t *offset, int32_t *perm, const int32_t *bigseg,
                                                      const int32_t *nbig)
{
    extern __shared__ int sm[];
    for (int e = blockIdx.x; e < *nbig; e += gridDim.x) {
    int cellk = bigseg[e];
    int start = offset[cellk];
    int m = offset[cellk + 1] - start;
    int32_t *seg = perm + start;
    bool in_smem = m <= SEG_BLOCK_MAX;
    int *s = in_smem ? sm : seg;
    if (in_smem) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = seg[i];
        __syncthreads();
    }
    int N = 1;
    while (N < m) N <<= 1;
    for (int k = 2; k <= N; k <<= 1) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            int l = i ^ (k - 1);
            if (l > i && l < m) {
                int a = s[i], b = s[l];
                if (b < a) { s[i] = b; s[l] = a; }
            }
        }
        __syncthreads();
        for (int j = k >> 2; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                int l = i ^ j;
                if (l > i && l < m) {
                    int a = s[i], b = s[l];
                    if (b < a) { s[i] = b; s[l] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (in_smem)
        for (int i = threadIdx.x; i < m; i += blockDim.x) seg[i] = s[i];
    __syncthreads();
    }
}

struct GatherArgs {
    int64_t nmax;
    const int32_t *live;  // offset[ncell] = number of live particles
    const int32_t *perm;
    const void *src[6];
    void *dst[6];
    const int32_t *cell_src;
    int32_t *cell_dst;
    const uint32_t *tag_src;
    uint32_t *tag_dst;
    int64_t *count_out;
};

template <typename T>
__global__ void gather_kernel(GatherArgs A, int nfields)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t live = *A.live;
    if (s == 0 && A.count_out) *A.count_out = live;
    if (s >= A.nmax) return;
    if (s < live) {
        int32_t src = A.perm[s];
        for (int k = 0; k < nfields; ++k) ((T *)A.dst[k])[s] = ((const T *)A.src[k])[src];
        A.tag_dst[s] = A.tag_src[src];
        if (A.cell_dst) A.cell_dst[s] = A.cell_src[src];
    } else {
        A.tag_dst[s] = DEAD;
    }
}

}  // namespace

cudaError_t sort_setup()
{
    return cudaFuncSetAttribute(bigseg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SEG_BLOCK_MAX * (int)sizeof(int));
}

cudaError_t launch_keys(grpic_ctx *ctx, const grpic_particles *p, cudaStream_t s)
{
    if (p->n <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((p->n + 255) / 256);
    if (ctx->prm.precision == 64)
        keys_kernel<true><<<blocks, 256, 0, s>>>(ctx->g, p->n, p->d_count, p->x1, p->x2, nullptr, p->tag, ctx->d_keys,
                                                 ctx->d_count);
    else
        keys_kernel<false><<<blocks, 256, 0, s>>>(ctx->g, p->n, p->d_count, nullptr, nullptr, p->cell, p->tag,
                                                  ctx->d_keys, ctx->d_count);
    return cudaGetLastError();
}

// Expects ctx->d_keys / ctx->d_count filled for the current order of *p.
cudaError_t launch_sort(grpic_ctx *ctx, grpic_particles *p, grpic_particles *q, cudaStream_t s)
{
    int ncell = ctx->g.nr * ctx->g.nth;
    int64_t nscan = (int64_t)ncell + 1;  // counts of every key incl. the dead one
    int nb = (int)((nscan + SCAN_TILE - 1) / SCAN_TILE);
    // offset[0..ncell] exclusive, offset[ncell+1] = total; live = offset[ncell]
    scan_tiles<<<nb, SCAN_T, 0, s>>>(ctx->d_count, ctx->d_offset, ctx->d_blocksum, nscan);
    scan_sums<<<1, SCAN_T, 0, s>>>(ctx->d_blocksum, nb, ctx->d_offset + nscan);
    add_back<<<(unsigned)((nscan + 255) / 256), 256, 0, s>>>(ctx->d_offset, ctx->d_blocksum, nscan);
    cudaMemsetAsync(ctx->d_cursor, 0, sizeof(int32_t) * nscan, s);
    int32_t *nbig = ctx->d_cursor + nscan;  // one extra int reserved after the cursors
    cudaMemsetAsync(nbig, 0, sizeof(int32_t), s);
    if (p->n > 0) {
        unsigned blocks = (unsigned)((p->n + 255) / 256);
        scatter_kernel<<<blocks, 256, 0, s>>>(p->n, p->d_count, ctx->d_keys, ctx->d_offset, ctx->d_cursor, ctx->d_perm,
                                              ncell);
    }
    segfix_kernel<<<(ncell + SEG_WARPS - 1) / SEG_WARPS, SEG_WARPS * 32, 0, s>>>(ctx->d_offset, ctx->d_perm, ncell,
                                                                                 ctx->d_bigseg, nbig, ctx->d_status);
    // oversized segments (rare): the list length is only known on the device,
    // so a fixed grid strides over it and returns at once when it is empty
    bigseg_kernel<<<64, 1024, SEG_BLOCK_MAX * sizeof(int), s>>>(ctx->d_offset, ctx->d_perm, ctx->d_bigseg, nbig);
    GatherArgs A;
    A.nmax = p->n;
    A.live = ctx->d_offset + ncell;
    A.perm = ctx->d_perm;
    A.tag_src = p->tag;
    A.tag_dst = q->tag;
    A.count_out = p->d_count;
    int nf = 5;
    void *sp[5] = {p->x1, p->x2, p->u1, p->u2, p->u3};
    void *dp[5] = {q->x1, q->x2, q->u1, q->u2, q->u3};
    for (int k = 0; k < 5; ++k) {
        A.src[k] = sp[k];
        A.dst[k] = dp[k];
    }
    A.src[5] = nullptr;
    A.dst[5] = nullptr;
    A.cell_src = (ctx->prm.precision == 32) ? p->cell : nullptr;
    A.cell_dst = (ctx->prm.precision == 32) ? q->cell : nullptr;
    if (p->n > 0) {
        unsigned blocks = (unsigned)((p->n + 255) / 256);
        if (ctx->prm.precision == 64)
            gather_kernel<double><<<blocks, 256, 0, s>>>(A, nf);
        else
            gather_kernel<float><<<blocks, 256, 0, s>>>(A, nf);
    }
    return cudaGetLastError();
}

}  // namespace grpic
