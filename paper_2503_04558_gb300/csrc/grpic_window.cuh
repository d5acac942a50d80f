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

// The 40 window values of one particle moving from (a1, a2) to (b1, b2), in
// cell units relative to the lower corner of its start cell (a in [0, 1],
// b in [-1, 2]); dphi its phi advance.  With CIC weights the prefix sums of
// Eq. esirkepov-decomp factor per dimension:
//   J^r A_r (k, l)     = -qw/(2dt) P_r(k) (S1_t + S0_t)(l),  P_r(k) = sum_{k'<=k} (S1_r - S0_r)(k')
//   J^th A_th (k, l)   = -qw/(2dt) (S1_r + S0_r)(k) P_t(l)
//   J^ph dV (k, l)     = qw dphi/dt (S1r S1t/3 + S1r S0t/6 + S0r S1t/6 + S0r S0t/3)(k, l)
// (Eq. j-phi-deposit), k, l = 0..3 standing for columns/rows -1..2.  The
// start point lies in its cell, so its weights are (0, 1 - a, a, 0) and
// only the end point's four weights per dimension need evaluating.
template <typename T>
__device__ __forceinline__ T cic_weight(T d)
{
    return fmax(T(0), T(1) - fabs(d));
}

template <typename T>
__device__ __forceinline__ void esirkepov_window(T a1, T a2, T b1, T b2, T qw, T dphi, T dt, T win[NWIN])
{
    const T S0r[4] = {T(0), T(1) - a1, a1, T(0)}, S0t[4] = {T(0), T(1) - a2, a2, T(0)};
    T S1r[4], S1t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        S1r[k] = cic_weight<T>(b1 - T(k - 1));
        S1t[k] = cic_weight<T>(b2 - T(k - 1));
    }
    const T cr = -qw / (T(2) * dt);
    const T cp = qw * dphi / dt;
    T Pr = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Pr += S1r[k] - S0r[k];
        const T c = cr * Pr;
#pragma unroll
        for (int l = 0; l < 4; ++l) win[k * 4 + l] = c * (S1t[l] + S0t[l]);
    }
    T Pt = T(0);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        Pt += S1t[l] - S0t[l];
        const T c = cr * Pt;
#pragma unroll
        for (int k = 0; k < 4; ++k) win[12 + k * 3 + l] = c * (S1r[k] + S0r[k]);
    }
    // J^phi = S1r (x) cp (S1t/3 + S0t/6) + S0r (x) cp (S1t/6 + S0t/3)
    T cU[4], cV[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        cU[l] = cp * (S1t[l] * (T(1) / T(3)) + S0t[l] * (T(1) / T(6)));
        cV[l] = cp * (S1t[l] * (T(1) / T(6)) + S0t[l] * (T(1) / T(3)));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) win[24 + k * 4 + l] = S1r[k] * cU[l] + S0r[k] * cV[l];
}

// Deposit of a warp's windows: the lanes are grouped by start cell and each
// group (up to MAXG of them; the usual warp after the sort has one or two)
// builds its windows and reduce-scatters them in turn, so every lane
// computes its window once and the 40 values live only here; lanes of the
// remaining groups add their own entries.  All 32 lanes must call.  (The
// FP64 push keeps its own deposit: on the FP64-bound kernel this grouping
// measured slower than reducing only warps with a single start cell.)
template <typename T, int MAXG>
__device__ __forceinline__ void deposit_warp(bool dep, int i0, int j0, int nr, T a1, T a2, T b1, T b2, T qw, T dphi,
                                             T dt, int lane, int nth, int ng, int64_t ld, T *J0, T *J1, T *J2)
{
    const unsigned FULL = 0xffffffffu;
    const int wk = dep ? j0 * nr + i0 : -1;
    bool pending = dep;
#pragma unroll 1
    for (int pass = 0; pass < MAXG; ++pass) {
        const unsigned todo = __ballot_sync(FULL, pending);
        if (!todo) return;
        const int leader = __ffs(todo) - 1;
        const int gk = __shfl_sync(FULL, wk, leader);
        const int gi = __shfl_sync(FULL, i0, leader), gj = __shfl_sync(FULL, j0, leader);
        const bool in = pending && wk == gk;
        T win[NWIN];
        if (in) {
            esirkepov_window<T>(a1, a2, b1, b2, qw, dphi, dt, win);
        } else {
#pragma unroll
            for (int v = 0; v < NWIN; ++v) win[v] = T(0);
        }
        T tot[2];
        int idx[2];
        window_reduce_scatter<T>(win, lane, tot, idx);
        window_add<T>(idx[0], tot[0], gi, gj, nth, ng, ld, J0, J1, J2);
        window_add<T>(idx[1], tot[1], gi, gj, nth, ng, ld, J0, J1, J2);
        pending = pending && !in;
    }
    if (pending) {
        T win[NWIN];
        esirkepov_window<T>(a1, a2, b1, b2, qw, dphi, dt, win);
#pragma unroll
        for (int v = 0; v < NWIN; ++v) window_add<T>(v, win[v], i0, j0, nth, ng, ld, J0, J1, J2);
    }
}

// The same deposit split by support.  A particle that stays in its start
// cell touches 8 window entries only (J^r A at face 1, rows 1-2; J^theta A at
// columns 1-2, face 1; J^phi dV at columns 1-2, rows 1-2): every lane adds its
// values at those 8 "core" entries into a warp reduction (grouped by start
// cell as above, 9 shuffles instead of 45), and a lane whose end point left
// the start cell (di, dj = floor(b) in -1..1 not both 0) adds its other
// nonzero entries directly: the extra column ex = 0 or 3 (face ef = 0 or 2)
// of an r move and the extra row of a theta move, 5 entries for a move along
// one axis, 13 for a diagonal one.  The entries and values are those of
// esirkepov_window; lanes that stay execute the extra part predicated off.
template <typename T>
__device__ __forceinline__ void reduce8(T v[8], int lane, T &tot, int &idx)
{
    const unsigned FULL = 0xffffffffu;
    int base = 0;
#pragma unroll
    for (int st = 0, half = 4, m = 16; st < 3; ++st, half >>= 1, m >>= 1) {
        const bool hi = lane & m;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < half) {
                T keep = hi ? v[k + half] : v[k];
                T send = hi ? v[k] : v[k + half];
                v[k] = keep + __shfl_xor_sync(FULL, send, m);
            }
        }
        base += hi ? half : 0;
    }
    v[0] += __shfl_xor_sync(FULL, v[0], 2);
    v[0] += __shfl_xor_sync(FULL, v[0], 1);
    tot = v[0];
    idx = (lane & 3) == 0 ? base : -1;  // one lane of each quad adds
}

// add v at window column k, row l of one current array (rows 0..rmax exist)
template <typename T>
__device__ __forceinline__ void add_at(T *J, int rmax, int i0, int j0, int k, int l, int ng, int64_t ld, T v)
{
    const int row = j0 - 1 + l;
    if (v == T(0) || row < 0 || row > rmax) return;
    atomicAdd(J + (size_t)row * ld + (i0 - 1 + k + ng), v);
}

// cr = -q w / (2 dt) and cq = q w / dt of the particle's species (the
// callers form them by multiplication with 1 / dt)
template <typename T, int MAXG>
__device__ __forceinline__ void deposit_warp_split(bool dep, int i0, int j0, int nr, T a1, T a2, T b1, T b2, T cr,
                                                   T cq, T dphi, int lane, int nth, int ng, int64_t ld, T *J0, T *J1,
                                                   T *J2)
{
    const unsigned FULL = 0xffffffffu;
    // per-dimension weights (k, l = 0..3 stand for columns / rows -1..2)
    T S1r[4], S1t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        S1r[k] = cic_weight<T>(b1 - T(k - 1));
        S1t[k] = cic_weight<T>(b2 - T(k - 1));
    }
    const T S0r1 = T(1) - a1, S0r2 = a1, S0t1 = T(1) - a2, S0t2 = a2;
    const T cp = cq * dphi;
    // prefix sums: Pr(k) = sum_{k' <= k} (S1r - S0r)(k'), Pt likewise
    const T Pr0 = S1r[0], Pr1 = Pr0 + S1r[1] - S0r1, Pr2 = Pr1 + S1r[2] - S0r2;
    const T Pt0 = S1t[0], Pt1 = Pt0 + S1t[1] - S0t1, Pt2 = Pt1 + S1t[2] - S0t2;
    const T S0t[4] = {T(0), S0t1, S0t2, T(0)}, S0r[4] = {T(0), S0r1, S0r2, T(0)};
    T cU[4], cV[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        cU[l] = cp * (S1t[l] * (T(1) / T(3)) + S0t[l] * (T(1) / T(6)));
        cV[l] = cp * (S1t[l] * (T(1) / T(6)) + S0t[l] * (T(1) / T(3)));
    }
    // ---- the 8 core entries, reduced per start-cell group
    const int wk = dep ? j0 * nr + i0 : -1;
    bool pending = dep;
#pragma unroll 1
    for (int pass = 0; pass < MAXG; ++pass) {
        const unsigned todo = __ballot_sync(FULL, pending);
        if (!todo) break;
        const int leader = __ffs(todo) - 1;
        const int gk = __shfl_sync(FULL, wk, leader);
        const int gi = __shfl_sync(FULL, i0, leader), gj = __shfl_sync(FULL, j0, leader);
        const bool in = pending && wk == gk;
        T v[8];
        if (in) {
            const T c1 = cr * Pr1;
            v[0] = c1 * (S1t[1] + S0t1);  // J^r A (face 1, row 1)
            v[1] = c1 * (S1t[2] + S0t2);  // J^r A (face 1, row 2)
            const T c2 = cr * Pt1;
            v[2] = c2 * (S1r[1] + S0r1);  // J^th A (column 1, face 1)
            v[3] = c2 * (S1r[2] + S0r2);  // J^th A (column 2, face 1)
            v[4] = S1r[1] * cU[1] + S0r1 * cV[1];  // J^ph (1, 1)
            v[5] = S1r[1] * cU[2] + S0r1 * cV[2];  // J^ph (1, 2)
            v[6] = S1r[2] * cU[1] + S0r2 * cV[1];  // J^ph (2, 1)
            v[7] = S1r[2] * cU[2] + S0r2 * cV[2];  // J^ph (2, 2)
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = T(0);
        }
        T tot;
        int idx;
        reduce8<T>(v, lane, tot, idx);
        if (idx >= 0) {
            // core entry idx: 0, 1 J^r A (face 1, rows 1, 2); 2, 3 J^th A
            // (columns 1, 2, face 1); 4..7 J^ph (columns 1, 2 x rows 1, 2)
            T *J = idx < 2 ? J0 : (idx < 4 ? J1 : J2);
            const int k = idx < 2 ? 1 : (idx < 4 ? idx - 1 : 1 + ((idx - 4) >> 1));
            const int l = idx < 2 ? 1 + idx : (idx < 4 ? 1 : 1 + ((idx - 4) & 1));
            add_at<T>(J, idx < 4 && idx >= 2 ? nth - 1 : nth, gi, gj, k, l, ng, ld, tot);
        }
        pending = pending && !in;
    }
    if (pending) {
        // lanes of start cells beyond MAXG groups: their core entries directly
        const T c1 = cr * Pr1, c2 = cr * Pt1;
        add_at<T>(J0, nth, i0, j0, 1, 1, ng, ld, c1 * (S1t[1] + S0t1));
        add_at<T>(J0, nth, i0, j0, 1, 2, ng, ld, c1 * (S1t[2] + S0t2));
        add_at<T>(J1, nth - 1, i0, j0, 1, 1, ng, ld, c2 * (S1r[1] + S0r1));
        add_at<T>(J1, nth - 1, i0, j0, 2, 1, ng, ld, c2 * (S1r[2] + S0r2));
        add_at<T>(J2, nth, i0, j0, 1, 1, ng, ld, S1r[1] * cU[1] + S0r1 * cV[1]);
        add_at<T>(J2, nth, i0, j0, 1, 2, ng, ld, S1r[1] * cU[2] + S0r1 * cV[2]);
        add_at<T>(J2, nth, i0, j0, 2, 1, ng, ld, S1r[2] * cU[1] + S0r2 * cV[1]);
        add_at<T>(J2, nth, i0, j0, 2, 2, ng, ld, S1r[2] * cU[2] + S0r2 * cV[2]);
    }
    // ---- the entries outside the core, lanes that left the start cell
    const int di = dep ? (int)floor(b1) : 0, dj = dep ? (int)floor(b2) : 0;
    if (!__any_sync(FULL, di != 0 || dj != 0)) return;
    const int ex = di > 0 ? 3 : 0, ef = di > 0 ? 2 : 0;  // extra column / face (valid if di != 0)
    const int ey = dj > 0 ? 3 : 0, eg = dj > 0 ? 2 : 0;  // extra row / theta face (valid if dj != 0)
    const T Prx = ef == 2 ? Pr2 : Pr0, Ptx = eg == 2 ? Pt2 : Pt0;
    const T S1rx = S1r[ex], S1tx = S1t[ey];
    if (di != 0) {
        // J^r A at the extra face, rows 1, 2; J^th A at the extra column,
        // face 1; J^ph at the extra column, rows 1, 2
        add_at<T>(J0, nth, i0, j0, ef, 1, ng, ld, cr * Prx * (S1t[1] + S0t1));
        add_at<T>(J0, nth, i0, j0, ef, 2, ng, ld, cr * Prx * (S1t[2] + S0t2));
        add_at<T>(J1, nth - 1, i0, j0, ex, 1, ng, ld, cr * S1rx * Pt1);
        add_at<T>(J2, nth, i0, j0, ex, 1, ng, ld, S1rx * cU[1]);
        add_at<T>(J2, nth, i0, j0, ex, 2, ng, ld, S1rx * cU[2]);
    }
    if (dj != 0) {
        // J^th A at the extra theta face, columns 1, 2; J^r A at face 1, the
        // extra row; J^ph at columns 1, 2, the extra row
        const T u3 = cp * S1tx * (T(1) / T(3)), u6 = cp * S1tx * (T(1) / T(6));
        add_at<T>(J1, nth - 1, i0, j0, 1, eg, ng, ld, cr * (S1r[1] + S0r1) * Ptx);
        add_at<T>(J1, nth - 1, i0, j0, 2, eg, ng, ld, cr * (S1r[2] + S0r2) * Ptx);
        add_at<T>(J0, nth, i0, j0, 1, ey, ng, ld, cr * Pr1 * S1tx);
        add_at<T>(J2, nth, i0, j0, 1, ey, ng, ld, S1r[1] * u3 + S0r1 * u6);
        add_at<T>(J2, nth, i0, j0, 2, ey, ng, ld, S1r[2] * u3 + S0r2 * u6);
    }
    if (di != 0 && dj != 0) {
        // the corner: J^r A (extra face, extra row), J^th A (extra column,
        // extra theta face), J^ph (extra column, extra row)
        add_at<T>(J0, nth, i0, j0, ef, ey, ng, ld, cr * Prx * S1tx);
        add_at<T>(J1, nth - 1, i0, j0, ex, eg, ng, ld, cr * S1rx * Ptx);
        add_at<T>(J2, nth, i0, j0, ex, ey, ng, ld, S1rx * cp * S1tx * (T(1) / T(3)));
    }
}

}  // namespace grpic
