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
//
// Neighbour sort (the step's sort when the particles are the output of the
// previous sort and one push moved them): a particle of old cell s lands in
// one of its 9 neighbours k = s + dj*n_r + di (di, dj in -1..1) or dies.  The
// stable order of cell k is then its sources in increasing cell order, each
// source's particles in slot order, so
//   6. count, per old cell, the particles going in each direction;
//   7. destination counts = sums over the 9 sources; exclusive scan;
//   8. each particle's slot index goes straight to offset[k] + (particles of
//      lower sources into k) + (its rank among its cell's particles in that
//      direction), with no atomics and no fix-up;
// and step 5's gather moves the data, as for the general path.  Placing only
// the indices keeps the per-cell bookkeeping off the particle data: the
// gather's reads are nearly sequential runs and its writes sequential.
// The count pass checks the precondition (every key a neighbour of its
// segment, live count = the previous sort's) and raises a device flag when
// it fails; the general kernels then run instead.  Every kernel of both paths
// reads the flag and strides over its work with a fixed grid, so the path
// not taken costs one flag read per block.
#include "grpic_internal.cuh"

#include <algorithm>
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
                if (r >= g.r_in && r < g.r_out && th >= 0.0 && th <= M_PI) {
                    // the cell the push would start from (x1 clamped into [0, nr))
                    int i = (int)floor((log(r) - g.ln_rin) / g.dx1);
                    i = i < 0 ? 0 : (i > g.nr - 1 ? g.nr - 1 : i);
                    int j = (int)floor(th / g.dth);
                    if (j > g.nth - 1) j = g.nth - 1;
                    key = j * g.nr + i;
                }
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

// general path kernels skip their work when flag is set and 0 (the neighbour
// sort applied); flag == nullptr always runs
__device__ __forceinline__ bool general_off(const int32_t *flag) { return flag && *flag == 0; }

__global__ void scatter_kernel(int64_t nmax, const int64_t *d_count, const int32_t *keys, const int32_t *offset,
                               int32_t *cursor, int32_t *perm, int ncell, const int32_t *flag)
{
    if (general_off(flag)) return;
    int64_t n = d_count ? *d_count : nmax;
    if (n > nmax) n = nmax;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t end = (n + 31) & ~(int64_t)31;  // whole warps take part in the match
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < end; p += stride) {
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
                                                                 int32_t *bigseg, int32_t *nbig, const int32_t *flag)
{
    if (general_off(flag)) return;
    __shared__ int sh[SEG_WARPS][SEG_WARP_MAX];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t cellk = (int64_t)blockIdx.x * SEG_WARPS + warp; cellk < ncell;
         cellk += (int64_t)gridDim.x * SEG_WARPS) {
        int start = offset[cellk];
        int m = offset[cellk + 1] - start;
        if (m <= 1) continue;
        int32_t *seg = perm + start;
        // already in order?  (the usual case for cells nobody entered)
        bool ok = true;
        for (int i = lane; i + 1 < m; i += 32) ok &= seg[i] <= seg[i + 1];
        if (__all_sync(0xffffffffu, ok)) continue;
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
            __syncwarp();
        } else if (lane == 0) {
            int k = atomicAdd(nbig, 1);
            bigseg[k] = (int32_t)cellk;
        }
    }
}

// one block per oversized segment: bitonic network in shared memory when it
// fits, in global memory otherwise
__global__ void __launch_bounds__(1024) bigseg_kernel(const int32_t *offset, int32_t *perm, const int32_t *bigseg,
                                                      const int32_t *nbig, const int32_t *flag)
{
    if (general_off(flag)) return;
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

// q[s] = p[perm[s]] for the live slots, DEAD tags past them.  Each thread
// moves four slots per round (their permutation entries first, then all
// their loads) so that enough loads are in flight to cover the latency.
template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(GatherArgs A, int nfields, const int32_t *flag)
{
    if (general_off(flag)) return;
    const int64_t live = *A.live;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s0 == 0 && A.count_out) *A.count_out = live;
    for (int64_t base = s0; base < A.nmax; base += 4 * stride) {
        int32_t src[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t s = base + u * stride;
            src[u] = s < live ? A.perm[s] : -1;
        }
        T v[4][5];
        uint32_t tg[4];
        int32_t cl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (src[u] < 0) continue;
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k < nfields) v[u][k] = ((const T *)A.src[k])[src[u]];
            tg[u] = A.tag_src[src[u]];
            if (A.cell_dst) cl[u] = A.cell_src[src[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t s = base + u * stride;
            if (s >= A.nmax) break;
            if (src[u] < 0) {
                A.tag_dst[s] = DEAD;
                continue;
            }
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k < nfields) ((T *)A.dst[k])[s] = v[u][k];
            A.tag_dst[s] = tg[u];
            if (A.cell_dst) A.cell_dst[s] = cl[u];
        }
    }
}

// histogram of existing keys (dead key included), for the general path
__global__ void hist_zero_kernel(int32_t *count, int64_t n, const int32_t *flag)
{
    if (general_off(flag)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        count[i] = 0;
}

__global__ void hist_kernel(int64_t nmax, const int64_t *d_count, const int32_t *keys, int32_t *count, int ncell,
                            const int32_t *flag)
{
    if (general_off(flag)) return;
    int64_t n = d_count ? *d_count : nmax;
    if (n > nmax) n = nmax;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t end = (n + 31) & ~(int64_t)31;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < end; p += stride) {
        int key = (p < n) ? keys[p] : -1;
        if (key > ncell) key = -1;
        unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
    }
}

// ---------------------------------------------------------------------------
// neighbour sort
// ---------------------------------------------------------------------------
// direction d = (dj+1)*3 + (di+1); cnt9 is stored direction-major (d*ncell + s)

// direction of key k from old cell s (column si): -1 if k is not one of the 9
// neighbours.  |k - s| <= n_r + 1 for a neighbour, and with n_r >= 3 the row
// step follows from the sign of k - s without a division.
__device__ __forceinline__ int dir_of(int k, int s, int si, int nr)
{
    int delta = k - s;
    int dj = (delta > 1) - (delta < -1);
    int di = delta - dj * nr;
    if (di < -1 || di > 1 || si + di < 0 || si + di >= nr) return -1;
    return (dj + 1) * 3 + (di + 1);
}

// The neighbour-sort passes walk the old cells in tasks of TASK_CELLS
// consecutive cells per warp: the task's particles [off[s0], off[s0 + m]) are
// one contiguous stream of 32-particle chunks (no pipeline restart at each
// cell), and a particle's old cell is found among the task's segment starts,
// which the lanes hold (lane l: off[s0 + l]).
constexpr int TASK_CELLS = 32;

// index (0 .. m-1) of the task cell whose segment holds slot b + lane: the
// number of segment starts off[s0 + l], 1 <= l < m, at or before it (empty
// segments share their start with the next one, so each counts).  A chunk
// rarely holds a segment start, so the starts inside it are visited one by
// one.  All 32 lanes call with the same b.
__device__ __forceinline__ int task_cell(int b, int lane, int o, int m)
{
    const unsigned FULL = 0xffffffffu;
    const bool own = lane >= 1 && lane < m;
    int c = __popc(__ballot_sync(FULL, own && o <= b));
    unsigned inside = __ballot_sync(FULL, own && o > b && o - b < 32);
    const int p = b + lane;
    while (inside) {
        const int l = __ffs(inside) - 1;
        inside &= inside - 1;
        c += p >= __shfl_sync(FULL, o, l);
    }
    return c;
}

// column of cell s0 + c given the column s0i of s0
__device__ __forceinline__ int task_col(int s0i, int c, int nr)
{
    int si = s0i + c;
    while (si >= nr) si -= nr;
    return si;
}

// step 6: per old cell s (segment [off[s], off[s+1]) of the previous sort's
// output), the particles moving in each direction; dead keys are dropped.
// Raises *flag if a key is not a neighbour or the live count changed.  Keys
// are loaded four chunks at a time (a short loop body needs the loads in
// flight to cover the memory latency).
__global__ void __launch_bounds__(256) count9_kernel(const int32_t *off, const int32_t *keys, int nr, int ncell,
                                                     const int64_t *d_count, int64_t nmax, int32_t *cnt9,
                                                     int32_t *flag)
{
    __shared__ int cnt_sh[8][TASK_CELLS * 9];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int *cnt = cnt_sh[wib];
    if (wid == 0 && lane == 0) {
        int64_t n = d_count ? *d_count : nmax;
        if (n != (int64_t)off[ncell] || n > nmax) atomicExch(flag, 1);
    }
    const int64_t ntask = ((int64_t)ncell + TASK_CELLS - 1) / TASK_CELLS;
    for (int64_t t = wid; t < ntask; t += nw) {
        const int64_t s0 = t * TASK_CELLS;
        const int m = (int)((int64_t)ncell - s0 < TASK_CELLS ? (int64_t)ncell - s0 : TASK_CELLS);
        const int o = off[s0 + (lane < m ? lane : m)];
        const int end = off[s0 + m];
        const int beg = __shfl_sync(FULL, o, 0);
        const int s0i = (int)(s0 % nr);
        for (int e = lane; e < TASK_CELLS * 9; e += 32) cnt[e] = 0;
        __syncwarp();
        bool bad = false;
        for (int b = beg; b < end; b += 4 * 32) {
            int kk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = b + u * 32 + lane;
                kk[u] = p < end ? keys[p] : -2;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = b + u * 32 + lane;
                if (b + u * 32 >= end) break;  // warp-uniform
                const int c = task_cell(b + u * 32, lane, o, m);
                int key2 = -1;
                if (p < end) {
                    const int k = kk[u];
                    if (k >= 0 && k < ncell) {
                        const int cls = dir_of(k, (int)(s0 + c), task_col(s0i, c, nr), nr);
                        bad |= cls < 0;
                        if (cls >= 0) key2 = c * 9 + cls;
                    } else {
                        bad |= k != ncell;
                    }
                }
                const unsigned peers = __match_any_sync(FULL, key2);
                if (key2 >= 0 && lane == __ffs(peers) - 1) cnt[key2] += __popc(peers);
                __syncwarp();
            }
        }
        if (lane < m)
#pragma unroll
            for (int d = 0; d < 9; ++d) cnt9[(int64_t)d * ncell + s0 + lane] = cnt[lane * 9 + d];
        if (__any_sync(FULL, bad) && lane == 0) atomicExch(flag, 1);
        __syncwarp();
    }
}

__device__ __forceinline__ int dir_di(int d) { return d % 3 - 1; }
__device__ __forceinline__ int dir_dj(int d) { return d / 3 - 1; }

// particles of direction d' arriving in cell (ik, jk), 0 if the source cell
// (ik - di', jk - dj') lies outside the grid
__device__ __forceinline__ int arrivals(const int32_t *cnt9, int nr, int nth, int64_t ncell, int ik, int jk, int d)
{
    int is = ik - dir_di(d), js = jk - dir_dj(d);
    if (is < 0 || is >= nr || js < 0 || js >= nth) return 0;
    return cnt9[(int64_t)d * ncell + (int64_t)js * nr + is];
}

// step 7: destination counts into count[] (count[ncell] = 0: the dead are dropped)
__global__ void dest_count_kernel(const int32_t *cnt9, int nr, int nth, int32_t *count, const int32_t *flag)
{
    if (*flag) return;
    const int64_t ncell = (int64_t)nr * nth;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= ncell;
         k += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        if (k < ncell) {
            int ik = (int)(k % nr), jk = (int)(k / nr);
#pragma unroll
            for (int d = 0; d < 9; ++d) c += arrivals(cnt9, nr, nth, ncell, ik, jk, d);
        }
        count[k] = c;
    }
}

// first destination slot of old cell s's direction-d particles:
// offset[k] + arrivals into k from the sources below s in cell order (the
// directions d' > d), k = s moved by d
__global__ void base9_kernel(const int32_t *cnt9, int32_t *base9, const int32_t *off_new, int nr, int nth,
                             const int32_t *flag)
{
    if (*flag) return;
    const int64_t ncell = (int64_t)nr * nth;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ncell; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)(s % nr), sj = (int)(s / nr);
        int base[9];
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            int ik = si + dir_di(d), jk = sj + dir_dj(d);
            int v = 0;
            if (ik >= 0 && ik < nr && jk >= 0 && jk < nth) {
                v = off_new[(int64_t)jk * nr + ik];
#pragma unroll
                for (int d2 = d + 1; d2 < 9; ++d2) v += arrivals(cnt9, nr, nth, ncell, ik, jk, d2);
            }
            base[d] = v;
        }
#pragma unroll
        for (int d = 0; d < 9; ++d) base9[(int64_t)d * ncell + s] = base[d];
    }
}


// step 8: stable placement of the indices: perm[dst] = src, the gather then
// moves the particle data (one pass with coalesced reads of nearly
// sequential runs).  A warp streams the keys of TASK_CELLS consecutive old
// cells; each particle takes the first free slot of its (old cell,
// direction) run (run counters in shared memory, started at base9), equal
// (cell, direction) lanes of a chunk taking consecutive slots in lane order.
__global__ void __launch_bounds__(256) neighbour_perm_kernel(const int32_t *off_old, const int32_t *base9,
                                                             const int32_t *keys, int nr, int nth, int64_t nmax,
                                                             int32_t *perm, const int32_t *flag)
{
    if (*flag) return;
    __shared__ int run_sh[8][TASK_CELLS * 9];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *run = run_sh[wib];
    const int64_t ncell = (int64_t)nr * nth;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntask = (ncell + TASK_CELLS - 1) / TASK_CELLS;
    for (int64_t t = wid; t < ntask; t += nw) {
        const int64_t s0 = t * TASK_CELLS;
        const int m = (int)(ncell - s0 < TASK_CELLS ? ncell - s0 : TASK_CELLS);
        const int o = off_old[s0 + (lane < m ? lane : m)];
        const int end = off_old[s0 + m];
        const int beg = __shfl_sync(FULL, o, 0);
        if (beg >= end) continue;  // warp-uniform
        if (lane < m)
#pragma unroll
            for (int d = 0; d < 9; ++d) run[lane * 9 + d] = base9[(int64_t)d * ncell + s0 + lane];
        __syncwarp();
        for (int b = beg; b < end; b += 4 * 32) {
            int kk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = b + u * 32 + lane;
                kk[u] = p < end ? keys[p] : -2;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (b + u * 32 >= end) break;  // warp-uniform
                const int p = b + u * 32 + lane;
                const int c = task_cell(b + u * 32, lane, o, m);
                const int k = kk[u];
                // the precondition holds here (checked by the count pass, or
                // by construction when the push counted: moves of at most one
                // cell), so the direction follows from k - s alone; a key out
                // of the 9 (never seen) is dropped rather than indexing run[]
                int key2 = -1;
                if (p < end && (unsigned)k < (unsigned)ncell) {
                    const int delta = k - (int)(s0 + c);
                    const int dj = (delta > 1) - (delta < -1);
                    const int di = delta - dj * nr;
                    if ((unsigned)(di + 1) <= 2u) key2 = c * 9 + (dj + 1) * 3 + (di + 1);
                }
                const unsigned peers = __match_any_sync(FULL, key2);
                const bool has = key2 >= 0;
                int dst = -1;
                if (has) dst = run[key2] + __popc(peers & ((1u << lane) - 1u));
                __syncwarp();
                if (has && lane == __ffs(peers) - 1) run[key2] += __popc(peers);
                __syncwarp();
                if ((uint64_t)(int64_t)dst < (uint64_t)nmax) perm[dst] = p;  // dst in [0, nmax)
            }
        }
        __syncwarp();
    }
}

}  // namespace

// exclusive scan of n int32 values into out[0..n) and their total into
// out[n]; bsum: SCAN_TILE scratch entries (n <= SCAN_TILE^2)
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int32_t *bsum, int64_t n, cudaStream_t s)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > SCAN_TILE) return cudaErrorInvalidValue;
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    scan_tiles<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, bsum, n);
    scan_sums<<<1, SCAN_T, 0, s>>>(bsum, (int)nb, out + n);
    add_back<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, bsum, n);
    return cudaGetLastError();
}

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
                                              ncell, nullptr);
    }
    segfix_kernel<<<(ncell + SEG_WARPS - 1) / SEG_WARPS, SEG_WARPS * 32, 0, s>>>(ctx->d_offset, ctx->d_perm, ncell,
                                                                                 ctx->d_bigseg, nbig, nullptr);
    // oversized segments (rare): the list length is only known on the device,
    // so a fixed grid strides over it and returns at once when it is empty
    bigseg_kernel<<<64, 1024, SEG_BLOCK_MAX * sizeof(int), s>>>(ctx->d_offset, ctx->d_perm, ctx->d_bigseg, nbig,
                                                                nullptr);
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
            gather_kernel<double><<<blocks, 256, 0, s>>>(A, nf, nullptr);
        else
            gather_kernel<float><<<blocks, 256, 0, s>>>(A, nf, nullptr);
    }
    return cudaGetLastError();
}

// The step's sort.  neighbour: the host's view allows the neighbour sort (the
// particles are the last sort's output and one push ran since); the device
// confirms it in the count pass.  Offsets of the result are left in
// ctx->d_offset (the previous ones are read from ctx->d_offset_prev).
cudaError_t launch_hist(grpic_ctx *ctx, const grpic_particles *p, cudaStream_t s)
{
    if (p->n <= 0) return cudaSuccess;
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->n + 255) / 256, (int64_t)dev_sms * 64));
    hist_kernel<<<g, 256, 0, s>>>(p->n, p->d_count, ctx->d_keys, ctx->d_count, ctx->g.nr * ctx->g.nth, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_sort_step(grpic_ctx *ctx, grpic_particles *p, grpic_particles *q, bool neighbour,
                             bool hist_on_fallback, bool materialize, bool counts_ready, cudaStream_t s)
{
    const int ncell = ctx->g.nr * ctx->g.nth;
    const int64_t nscan = (int64_t)ncell + 1;
    const int nb = (int)((nscan + SCAN_TILE - 1) / SCAN_TILE);
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned grid = (unsigned)dev_sms * 8;  // fixed grids, strided work
    int32_t *flag = ctx->d_sortflag;
    if (neighbour && ctx->g.nr >= 3) {
        cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
        // (a push that read through the last sort's permutation counted
        // already: its slots are that sort's segments by construction)
        if (!counts_ready)
            count9_kernel<<<grid, 256, 0, s>>>(ctx->d_offset_prev, ctx->d_keys, ctx->g.nr, ncell, p->d_count, p->n,
                                               ctx->d_cnt9, flag);
        dest_count_kernel<<<grid, 256, 0, s>>>(ctx->d_cnt9, ctx->g.nr, ctx->g.nth, ctx->d_count, flag);
        if (hist_on_fallback) {
            // the push skipped the histogram: rebuild it if the device fell back
            hist_zero_kernel<<<grid, 256, 0, s>>>(ctx->d_count, nscan, flag);
            hist_kernel<<<grid, 256, 0, s>>>(p->n, p->d_count, ctx->d_keys, ctx->d_count, ncell, flag);
        }
    } else {
        cudaMemsetAsync(flag, 0xff, sizeof(int32_t), s);  // nonzero: general path
    }
    // d_count holds the destination counts (neighbour path) or the push's
    // histogram (general path); one scan serves both
    scan_tiles<<<nb, SCAN_T, 0, s>>>(ctx->d_count, ctx->d_offset, ctx->d_blocksum, nscan);
    scan_sums<<<1, SCAN_T, 0, s>>>(ctx->d_blocksum, nb, ctx->d_offset + nscan);
    add_back<<<(unsigned)((nscan + 255) / 256), 256, 0, s>>>(ctx->d_offset, ctx->d_blocksum, nscan);
    if (neighbour && ctx->g.nr >= 3 && p->n > 0) {
        base9_kernel<<<grid, 256, 0, s>>>(ctx->d_cnt9, ctx->d_base9, ctx->d_offset, ctx->g.nr, ctx->g.nth, flag);
        neighbour_perm_kernel<<<grid, 256, 0, s>>>(ctx->d_offset_prev, ctx->d_base9, ctx->d_keys, ctx->g.nr,
                                                   ctx->g.nth, p->n, ctx->d_perm, flag);
    }
    // general path to the permutation (skipped on the device when the neighbour sort applied)
    cudaMemsetAsync(ctx->d_cursor, 0, sizeof(int32_t) * nscan, s);
    int32_t *nbig = ctx->d_cursor + nscan;
    cudaMemsetAsync(nbig, 0, sizeof(int32_t), s);
    // general path grids: enough blocks for memory parallelism, few enough
    // that skipping them costs little
    const int64_t gmax = (int64_t)dev_sms * 64;
    const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->n + 255) / 256, gmax));
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ncell + SEG_WARPS - 1) / SEG_WARPS, gmax));
    if (p->n > 0)
        scatter_kernel<<<gp, 256, 0, s>>>(p->n, p->d_count, ctx->d_keys, ctx->d_offset, ctx->d_cursor, ctx->d_perm,
                                          ncell, flag);
    segfix_kernel<<<gs, SEG_WARPS * 32, 0, s>>>(ctx->d_offset, ctx->d_perm, ncell, ctx->d_bigseg, nbig, flag);
    bigseg_kernel<<<64, 1024, SEG_BLOCK_MAX * sizeof(int), s>>>(ctx->d_offset, ctx->d_perm, ctx->d_bigseg, nbig, flag);
    GatherArgs G;
    G.nmax = p->n;
    G.live = ctx->d_offset + ncell;
    G.perm = ctx->d_perm;
    G.tag_src = p->tag;
    G.tag_dst = q->tag;
    G.count_out = p->d_count;
    void *sp[5] = {p->x1, p->x2, p->u1, p->u2, p->u3};
    void *dp[5] = {q->x1, q->x2, q->u1, q->u2, q->u3};
    for (int k = 0; k < 5; ++k) {
        G.src[k] = sp[k];
        G.dst[k] = dp[k];
    }
    G.src[5] = nullptr;
    G.dst[5] = nullptr;
    G.cell_src = (ctx->prm.precision == 32) ? p->cell : nullptr;
    G.cell_dst = (ctx->prm.precision == 32) ? q->cell : nullptr;
    // both paths leave the permutation in d_perm: one gather moves the data
    // (or the next push reads through it)
    if (p->n > 0 && materialize) {
        if (ctx->prm.precision == 64)
            gather_kernel<double><<<gp, 256, 0, s>>>(G, 5, nullptr);
        else
            gather_kernel<float><<<gp, 256, 0, s>>>(G, 5, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace grpic
