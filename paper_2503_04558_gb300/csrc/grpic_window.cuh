// grpic_window.cuh -- the warp's share of the Esirkepov current deposit
// (Sec. 2.3, Eq. esirkepov-decomp) with cloud-in-cell weights, for warps
// whose lanes mostly start in one cell (the usual case after the sort by
// cell).
//
// A particle's window spans columns i0-1..i0+2 and rows j0-1..j0+2 of its
// start cell (i0, j0): J^r A_r at 3x4 faces, J^theta A_theta at 4x3 faces and
// J^phi dV at 4x4 vertices.  With CIC weights the prefix sums of Eq.
// esirkepov-decomp factor per dimension:
//   J^r A_r (k, l)   = -qw/(2dt) P_r(k) (S1_t + S0_t)(l),  P_r(k) = sum_{k'<=k} (S1_r - S0_r)(k')
//   J^th A_th (k, l) = -qw/(2dt) (S1_r + S0_r)(k) P_t(l)
//   J^ph dV (k, l)   = qw dphi/dt (S1r S1t/3 + S1r S0t/6 + S0r S1t/6 + S0r S0t/3)(k, l)
// (Eq. j-phi-deposit), k, l = 0..3 standing for columns/rows -1..2.  The
// start point lies in its cell, so its weights are (0, 1 - a, a, 0).
#pragma once

#include <cuda_runtime.h>

namespace grpic {

// cloud-in-cell weight of a node at signed distance d (cells)
template <typename T>
__device__ __forceinline__ T cic_weight(T d)
{
    return fmax(T(0), T(1) - fabs(d));
}

// The deposit split by support.  A particle that stays in its start cell
// touches 8 window entries only (J^r A at face 1, rows 1-2; J^theta A at
// columns 1-2, face 1; J^phi dV at columns 1-2, rows 1-2): the lanes of each
// start cell (a group; the usual warp after the sort has one or two) reduce
// their values at those 8 "core" entries across the warp -- recursive
// halving over lane bits 4, 3, 2 (8 -> 4 -> 2 -> 1 values per lane, each lane
// keeping the half its bit selects and adding its partner's copy) and a
// butterfly over bits 1, 0: 9 shuffles -- and one lane of each quad adds a
// total.  A lane whose end point left the start cell (di, dj = floor(b) in
// -1..1 not both 0) adds its other nonzero entries directly: the extra column
// ex = 0 or 3 (face ef = 0 or 2) of an r move and the extra row of a theta
// move, 5 entries for a move along one axis, 13 for a diagonal one.  Lanes
// that stay execute the extra part predicated off.
// cr = -q w / (2 dt) and cq = q w / dt of the particle's species (the
// callers form them by multiplication with 1 / dt).  The end point b lies in
// [-1, 2) per dimension (a move of less than one cell; the push reflects it
// at the axis), so the core rows j0, j0+1 exist in every current array (J^r,
// J^phi rows 0..n_theta, J^theta rows 0..n_theta-1) and an extra row j0-1 or
// j0+2 is skipped where it does not (its entries are then zero: an end point
// on theta = pi exactly has b2 = 1).  Element offsets are 32-bit
// ((n_theta + 1) ld < 2^31).
template <typename T, int MAXG>
__device__ __forceinline__ void deposit_warp_split(bool dep, int i0, int j0, int nr, T a1, T a2, T b1, T b2, T cr,
                                                   T cq, T dphi, int lane, int nth, int ng, int ld, T *J0, T *J1,
                                                   T *J2)
{
    const unsigned FULL = 0xffffffffu;
    // end-point weights at columns / rows -1..2 for b in [-1, 2)
    const T S1r0 = fmax(T(0), -b1), S1r1 = fmax(T(0), T(1) - fabs(b1)), S1r2 = fmax(T(0), T(1) - fabs(b1 - T(1))),
            S1r3 = fmax(T(0), b1 - T(1));
    const T S1t0 = fmax(T(0), -b2), S1t1 = fmax(T(0), T(1) - fabs(b2)), S1t2 = fmax(T(0), T(1) - fabs(b2 - T(1))),
            S1t3 = fmax(T(0), b2 - T(1));
    const T S0r1 = T(1) - a1, S0r2 = a1, S0t1 = T(1) - a2, S0t2 = a2;
    const T cp = cq * dphi;
    // prefix sums P(k) = sum_{k' <= k} (S1 - S0)(k'); both weight sets sum to
    // one, so P(2) = -S1(3)
    const T Pr0 = S1r0, Pr1 = Pr0 + S1r1 - S0r1, Pr2 = -S1r3;
    const T Pt0 = S1t0, Pt1 = Pt0 + S1t1 - S0t1, Pt2 = -S1t3;
    // J^phi weights along theta: cU = cp (S1t/3 + S0t/6), cV = cp (S1t/6 + S0t/3)
    const T cp3 = cp * (T(1) / T(3)), cp6 = cp * (T(1) / T(6));
    const T cU1 = S1t1 * cp3 + S0t1 * cp6, cU2 = S1t2 * cp3 + S0t2 * cp6;
    const T cV1 = S1t1 * cp6 + S0t1 * cp3, cV2 = S1t2 * cp6 + S0t2 * cp3;
    // ---- the 8 core entries (columns / rows 1, 2 of the window), reduced per
    // start-cell group: J^r A (face 1, rows 1, 2), J^th A (columns 1, 2, face
    // 1), J^ph dV (columns 1, 2 x rows 1, 2)
    const T c1 = cr * Pr1, c2 = cr * Pt1;
    const T core[8] = {c1 * (S1t1 + S0t1), c1 * (S1t2 + S0t2), c2 * (S1r1 + S0r1), c2 * (S1r2 + S0r2),
                       S1r1 * cU1 + S0r1 * cV1, S1r1 * cU2 + S0r1 * cV2, S1r2 * cU1 + S0r2 * cV1,
                       S1r2 * cU2 + S0r2 * cV2};
    // after the reduction lane (lane & 3) == 0 holds the total of core entry
    // (lane >> 2) & 7: its array and its offset from the group's cell
    const int e = (lane >> 2) & 7;
    T *const Je = e < 2 ? J0 : (e < 4 ? J1 : J2);
    const int ek = e < 2 ? 0 : (e < 4 ? e - 2 : (e - 4) >> 1);  // column - 1
    const int el = e < 2 ? e : (e < 4 ? 0 : (e - 4) & 1);       // row - 1
    const int eoff = el * ld + ek + ng;
    const bool adder = (lane & 3) == 0;
    const int wk = dep ? j0 * nr + i0 : -1;
    const int wc = j0 * ld + i0;  // the start cell's element offset (without the guard columns)
    bool pending = dep;
#pragma unroll 1
    for (int pass = 0; pass < MAXG; ++pass) {
        const unsigned todo = __ballot_sync(FULL, pending);
        if (!todo) break;
        const int leader = __ffs(todo) - 1;
        const int gk = __shfl_sync(FULL, wk, leader);
        const int gc = __shfl_sync(FULL, wc, leader);
        const bool in = pending && wk == gk;
        T v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = in ? core[k] : T(0);
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
        }
        v[0] += __shfl_xor_sync(FULL, v[0], 2);
        v[0] += __shfl_xor_sync(FULL, v[0], 1);
        if (adder) atomicAdd(Je + (gc + eoff), v[0]);
        pending = pending && !in;
    }
    const int w11 = wc + ng;  // offset of the start cell's own node (window column 1, row 1)
    if (pending) {
        // lanes of start cells beyond MAXG groups: their core entries directly
        atomicAdd(J0 + w11, core[0]);
        atomicAdd(J0 + (w11 + ld), core[1]);
        atomicAdd(J1 + w11, core[2]);
        atomicAdd(J1 + (w11 + 1), core[3]);
        atomicAdd(J2 + w11, core[4]);
        atomicAdd(J2 + (w11 + ld), core[5]);
        atomicAdd(J2 + (w11 + 1), core[6]);
        atomicAdd(J2 + (w11 + ld + 1), core[7]);
    }
    // ---- the entries outside the core, lanes that left the start cell
    const int di = dep ? (int)floor(b1) : 0, dj = dep ? (int)floor(b2) : 0;
    if (!__any_sync(FULL, di != 0 || dj != 0)) return;
    // extra column ex = 0 or 3 / face ef = 0 or 2 of an r move, extra row ey
    // = 0 or 3 / theta face eg = 0 or 2 of a theta move, as offsets from the
    // core: column ex - 1 = -1 or 2, face ef - 1 = -1 or 1, rows likewise
    const int cx = di > 0 ? 2 : -1, cf = di > 0 ? 1 : -1;
    const int ry = (dj > 0 ? 2 : -1) * ld, rg = (dj > 0 ? 1 : -1) * ld;
    const T Prx = di > 0 ? Pr2 : Pr0, Ptx = dj > 0 ? Pt2 : Pt0;
    const T S1rx = di > 0 ? S1r3 : S1r0, S1tx = dj > 0 ? S1t3 : S1t0;
    const bool row_ok = dj > 0 ? j0 + 2 <= nth : j0 >= 1;  // the extra row exists
    if (di != 0) {
        // J^r A at the extra face, rows 1, 2; J^th A at the extra column,
        // face 1; J^ph at the extra column, rows 1, 2
        atomicAdd(J0 + (w11 + cf), cr * Prx * (S1t1 + S0t1));
        atomicAdd(J0 + (w11 + ld + cf), cr * Prx * (S1t2 + S0t2));
        atomicAdd(J1 + (w11 + cx), cr * S1rx * Pt1);
        atomicAdd(J2 + (w11 + cx), S1rx * cU1);
        atomicAdd(J2 + (w11 + ld + cx), S1rx * cU2);
    }
    if (dj != 0 && row_ok) {
        // J^th A at the extra theta face, columns 1, 2; J^r A at face 1, the
        // extra row; J^ph at columns 1, 2, the extra row
        const T u3 = cp3 * S1tx, u6 = cp6 * S1tx;
        atomicAdd(J1 + (w11 + rg), cr * (S1r1 + S0r1) * Ptx);
        atomicAdd(J1 + (w11 + rg + 1), cr * (S1r2 + S0r2) * Ptx);
        atomicAdd(J0 + (w11 + ry), cr * Pr1 * S1tx);
        atomicAdd(J2 + (w11 + ry), S1r1 * u3 + S0r1 * u6);
        atomicAdd(J2 + (w11 + ry + 1), S1r2 * u3 + S0r2 * u6);
    }
    if (di != 0 && dj != 0 && row_ok) {
        // the corner: J^r A (extra face, extra row), J^th A (extra column,
        // extra theta face), J^ph (extra column, extra row)
        atomicAdd(J0 + (w11 + ry + cf), cr * Prx * S1tx);
        atomicAdd(J1 + (w11 + rg + cx), cr * S1rx * Ptx);
        atomicAdd(J2 + (w11 + ry + cx), S1rx * cp3 * S1tx);
    }
}

}  // namespace grpic
