// grpic_window.cuh -- warp reduction of the 4x4 Esirkepov current window
// (Sec. 2.3, Eq. esirkepov-decomp) when all 32 lanes of a warp start in one
// cell (the usual case after the sort by cell).
//
// The window holds 40 values: J^r A_r at 3x4 faces (index k*4 + l), J^theta
// A_theta at 4x3 faces (12 + k*3 + l) and J^phi dV at 4x4 vertices
// (24 + k*4 + l), k = column offset - 1 + i0, l = row offset - 1 + j0.
// Recursive halving over lane bits 4, 3, 2 splits the 40 values into halves
// (40 -> 20 -> 10 -> 5), each lane keeping the half its bit selects and
// adding its partner's copy of it; a butterfly over bits 1, 0 then totals the
// remaining 5 within each quad, and the quad's lanes share out the 5 totals.
// 45 shuffles and 45 adds per lane instead of 200 each for a full butterfly
// of every value, and the atomics are spread over all lanes.
#pragma once

#include <cuda_runtime.h>

namespace grpic {

constexpr int NWIN = 40;

// on return lane holds the totals of window entries idx[0], idx[1] in out[];
// idx = -1 marks an unused slot
template <typename T>
__device__ __forceinline__ void window_reduce_scatter(T win[NWIN], int lane, T out[2], int idx[2])
{
    const unsigned FULL = 0xffffffffu;
    int base = 0;
    {
        const bool hi = (lane >> 4) & 1;
#pragma unroll
        for (int v = 0; v < 20; ++v) {
            T keep = hi ? win[v + 20] : win[v];
            T send = hi ? win[v] : win[v + 20];
            win[v] = keep + __shfl_xor_sync(FULL, send, 16);
        }
        base += hi ? 20 : 0;
    }
    {
        const bool hi = (lane >> 3) & 1;
#pragma unroll
        for (int v = 0; v < 10; ++v) {
            T keep = hi ? win[v + 10] : win[v];
            T send = hi ? win[v] : win[v + 10];
            win[v] = keep + __shfl_xor_sync(FULL, send, 8);
        }
        base += hi ? 10 : 0;
    }
    {
        const bool hi = (lane >> 2) & 1;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            T keep = hi ? win[v + 5] : win[v];
            T send = hi ? win[v] : win[v + 5];
            win[v] = keep + __shfl_xor_sync(FULL, send, 4);
        }
        base += hi ? 5 : 0;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        win[v] += __shfl_xor_sync(FULL, win[v], 2);
        win[v] += __shfl_xor_sync(FULL, win[v], 1);
    }
    const int q = lane & 3;  // quad lane: 0 -> entries 0, 1; 1 -> 2; 2 -> 3; 3 -> 4
    T a = win[0], b = win[1];
    if (q == 1) a = win[2];
    if (q == 2) a = win[3];
    if (q == 3) a = win[4];
    out[0] = a;
    out[1] = b;
    idx[0] = base + (q == 0 ? 0 : q + 1);
    idx[1] = (q == 0) ? base + 1 : -1;
}

// add one window entry v of the start cell (i0, j0) into the integrated
// currents (row ranges as in the deposit: J^r, J^phi rows 0..nth, J^theta
// rows 0..nth-1; column i0 - 1 + k plus the guard offset ng)
template <typename T>
__device__ __forceinline__ void window_add(int v, T val, int i0, int j0, int nth, int ng, int64_t ld, T *J0, T *J1,
                                           T *J2)
{
    if (v < 0 || val == T(0)) return;
    T *dst;
    int k, l, rmax;
    if (v < 12) {
        k = v >> 2;
        l = v & 3;
        dst = J0;
        rmax = nth;
    } else if (v < 24) {
        k = (v - 12) / 3;
        l = (v - 12) - 3 * k;
        dst = J1;
        rmax = nth - 1;
    } else {
        k = (v - 24) >> 2;
        l = (v - 24) & 3;
        dst = J2;
        rmax = nth;
    }
    int row = j0 - 1 + l;
    if (row < 0 || row > rmax) return;
    atomicAdd(dst + (size_t)row * ld + (i0 - 1 + k + ng), val);
}

}  // namespace grpic
