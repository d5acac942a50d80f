// grpic_internal.cuh -- context layout and device math shared by the CUDA
// translation units of libgrpic (sm_103a).
//
// Kerr-Schild 3+1 quantities follow App. A of arXiv:2503.04558 (Eqs.
// ks-coefficients, ks-variables, gamma-inverse, ks-alpha-beta).  The
// determinant is used in its closed form sqrt(gamma) = rho^2 sin(theta)
// sqrt(1+z) (from sqrt(-g) = rho^2 sin(theta) = alpha sqrt(gamma)).
#pragma once

#include <vector>

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/grpic.h"

namespace grpic {

constexpr int NG = 2;                   // guard columns on each side in r
constexpr uint32_t DEAD = 0x80000000u;  // tag bit of a dead particle
constexpr int NGL = 10;                 // Gauss-Legendre points per dimension

// Table slots (each (n_theta+1) x ld_tab doubles).
enum TabSlot {
    T_INV_ADR = 0, T_INV_ADT, T_INV_ADP, T_INV_ABR, T_INV_ABT, T_INV_ABP,
    T_ADR, T_ADT, T_ADP, T_ABR, T_ABT, T_ABP,
    T_AGRR_DR, T_AGRP_DR,            // at D^r   (i+1/2, j)
    T_AGTT_DT, T_SGB_DT,             // at D^th  (i, j+1/2)
    T_AGPP_DP, T_AGRP_DP, T_SGB_DP,  // at D^ph  (i, j)
    T_AGRR_BR, T_AGRP_BR,            // at B^r   (i, j+1/2)
    T_AGTT_BT, T_SGB_BT,             // at B^th  (i+1/2, j)
    T_AGPP_BP, T_AGRP_BP, T_SGB_BP,  // at B^ph  (i+1/2, j+1/2)
    T_COUNT
};

struct GridDev {
    int nr, nth, ld_tab;
    double a, r_in, r_out, dx1, dth, ln_rin;
};

}  // namespace grpic

struct grpic_ctx {
    int device;
    grpic_grid grid;
    grpic_params prm;
    grpic::GridDev g;
    double gl_x[grpic::NGL], gl_w[grpic::NGL];
    // device tables (FP64) and their FP32 copies
    double *tab;        // T_COUNT slabs
    double *col1d;      // per column: dr_prim, dr_dual, damp_int, damp_half (4 x ld_tab)
    float *tab32;       // FP32 copies of tab (precision 32 only)
    float *col1d32;
    size_t slab;        // elements per slab = (nth+1)*ld_tab
    double *rcol;       // r at integer columns r_in exp(i dx1), index i + NG
    float *rcol2;       // the same as (hi, lo) float pairs (precision 32 only)
    float *rowsc;       // sin, cos of theta_j = j dtheta as (hi, lo) pairs, j = 0..nth (precision 32)
    // field-solver scratch: Cn[6], two iterate buffers[12] in field precision
    void *fscratch;
    int64_t fscratch_ld;
    // status word and sort scratch
    int *d_status;
    int32_t *d_keys;      // per particle key of the last push
    int64_t keys_cap;
    int32_t *d_count;     // ncells+1 histogram
    int32_t *d_offset;    // ncells+2 exclusive scan
    int32_t *d_cursor;    // ncells+1 running fill
    int32_t *d_blocksum;  // scan partials
    int32_t *d_perm;      // new slot -> old slot
    int32_t *d_bigseg;    // list of oversized segments
    int32_t *d_offset_prev;  // segment offsets of the last sort's output (ncell+3)
    int32_t *d_cnt9;      // per old cell, particles moving in each of 9 directions (9 x ncell)
    int32_t *d_base9;     // per old cell and direction, the first destination slot (9 x ncell)
    int32_t *d_sortflag;  // 0: neighbour sort applies, 1: general counting sort
    const uint32_t *sorted_tag;  // tag array the last sort wrote
    int64_t pushes_since_sort;
    // a sort inside grpic_step that left its order in d_perm for the next
    // push to read through (the data in the tag array pending_tag unmoved)
    int pending_perm;
    const uint32_t *pending_tag;
    int counts_ready;  // the last (permuted) push filled d_cnt9 for the next sort
    // 2D radiation and injection: per-slot spawn counts, block sums/offsets,
    // charged particles and injection flags per cell; q/m and massive per
    // species on the device
    int32_t *d_spawn, *d_rad;
    int64_t rad_cap;
    double *d_spqm;
    int *d_spmassive;
    int64_t perm_cap;
    int keys_valid;       // keys of the current order are valid
    int hist_valid;       // and so is their histogram (d_count)
    const uint32_t *keys_tag;  // tag array of the particles those keys belong to
    int64_t step_count;
    // CUDA graph of two steps (grpic_step_graph) and the buffers it was captured on
    cudaStream_t cap_stream;
    cudaGraphExec_t graph_exec;
    const void *graph_key[24];
    int32_t *graph_offset;     // d_offset when the graph was captured (its double buffer's phase)
    // phase timing of grpic_step: 4 events per timed step (before the push,
    // after it, after the field update, after the sort)
    int timing;
    std::vector<cudaEvent_t> *tevents;
    int64_t tsteps;
    // FP32 field update by fused shared-memory launches (1, the default) or
    // one launch per stage (0); grpic_set_field_path
    int field_fused;
    // grpic_step_host: copy streams (host to device, device to host), one
    // event per copy chunk, and a pinned word for the live count
    cudaStream_t up_stream, down_stream;
    std::vector<cudaEvent_t> *hevents;
    int64_t *h_count;
    // FP32 form: the field components as float4 quads of the push's bilinear
    // stencils (launch_quad32, before each push), 6 x (nth+1) x fscratch_ld,
    // allocated with the field scratch
    void *q32;
    char err[256];
};

namespace grpic {

// ---------------------------------------------------------------------------
// Kerr-Schild geometry on the device.
// ---------------------------------------------------------------------------
struct KS {
    double alpha, beta;                 // lapse, radial shift
    double g_rr, g_rp, g_tt, g_pp;      // gamma_ij  (t = theta)
    double gi_rr, gi_rp, gi_tt, gi_pp;  // gamma^ij
    double sqrtg;
};

__host__ __device__ inline void ks_point(double a, double r, double th, KS &m)
{
    double s, c;
#ifdef __CUDA_ARCH__
    sincos(th, &s, &c);
#else
    s = std::sin(th);
    c = std::cos(th);
#endif
    double s2 = s * s, a2 = a * a;
    double rho2 = r * r + a2 * c * c;
    double irho2 = 1.0 / rho2;
    double z = 2.0 * r * irho2;
    double opz = 1.0 + z;
    double iopz = 1.0 / opz;
    double Dl = r * r + a2 - 2.0 * r;
    double Sg = (r * r + a2) * (r * r + a2) - a2 * Dl * s2;
    m.alpha = sqrt(iopz);
    m.beta = z * iopz;
    m.g_rr = opz;
    m.g_tt = rho2;
    m.g_pp = Sg * s2 * irho2;
    m.g_rp = -a * s2 * opz;
    m.gi_rr = (a2 + r * r) * irho2 - m.beta;
    m.gi_rp = a * irho2;
    m.gi_tt = irho2;
    m.gi_pp = irho2 / s2;
    m.sqrtg = rho2 * s * sqrt(opz);
}

__host__ __device__ inline double ks_sqrtg(double a, double r, double th)
{
    double s, c;
#ifdef __CUDA_ARCH__
    sincos(th, &s, &c);
#else
    s = std::sin(th);
    c = std::cos(th);
#endif
    double rho2 = r * r + a * a * c * c;
    return rho2 * s * sqrt(1.0 + 2.0 * r / rho2);
}

__host__ __device__ inline double r_of(const GridDev &g, double x1) { return g.r_in * exp(x1 * g.dx1); }

__device__ inline void set_status(int *st, int code) { atomicCAS(st, 0, code); }

// Record of one FP64 push kept for the adjoint (structure of arrays: entry k
// of particle p at tape[k * tape_ld + p]):
//   TAPE_U + 0..2    u' after the Boris step (u itself for an uncharged particle)
//   TAPE_SC0 + 0..1  sin, cos of theta^n
//   TAPE_IT + 6 it   the point of corrector `it`'s right-hand side (it < n_iter):
//                    r, theta, u_r, u_theta, sin theta, cos theta
//   tape_end(n)      x^{n+1} before the axis reflection: r, theta, u_r, u_theta,
//                    then delta phi
// Written for every particle the push moved or refused after the geodesic step.
constexpr int TAPE_U = 0, TAPE_SC0 = 3, TAPE_IT = 5;
__host__ __device__ constexpr int tape_end(int n_iter) { return TAPE_IT + 6 * n_iter; }
__host__ __device__ constexpr int tape_width(int n_iter) { return tape_end(n_iter) + 5; }

}  // namespace grpic

// entry points implemented in the kernel translation units (host side)
namespace grpic {
cudaError_t launch_tables(grpic_ctx *ctx, cudaStream_t s);
cudaError_t launch_init_fields(grpic_ctx *ctx, int kind, double B0, const grpic_fields *f, cudaStream_t s);
// push (fused with the deposit) of the particles of `in` into `p`: in place
// when perm is null (in == p), else slot k of p takes the particle of slot
// perm[k] of in for k < *live (the last sort's permutation, data not moved)
// and, when cnt9 is given (zeroed), the push also counts per start cell and
// direction for the next neighbour sort
// slot0: the first slot of the arrays given (a chunk of the slot range: the
// keys are written from d_keys + slot0)
cudaError_t launch_push64(grpic_ctx *ctx, const grpic_particles *in, grpic_particles *p, const int32_t *perm,
                          const int32_t *live, int32_t *cnt9, grpic_fields *f, bool histogram, cudaStream_t s,
                          int64_t slot0 = 0);
// the FP64 push in place, writing the adjoint's record of every particle
// (layout above, tape_ld >= p->n)
cudaError_t launch_push64_tape(grpic_ctx *ctx, grpic_particles *p, grpic_fields *f, double *tape, int64_t tape_ld,
                               cudaStream_t s);
// the FP32 push reads the fields through their stencil quads (ctx->q32),
// which launch_quad32 builds from f; launch it after every change of D, B
// and before the push (both fail with cudaErrorInvalidValue unless the field
// scratch is allocated for f->ld).  On the way it zeroes f->J (zero_j) and
// the 9 x n_cells counts zero_cnt9 (if not null).
cudaError_t launch_quad32(grpic_ctx *ctx, grpic_fields *f, bool zero_j, int32_t *zero_cnt9, cudaStream_t s);
cudaError_t launch_push32(grpic_ctx *ctx, const grpic_particles *in, grpic_particles *p, const int32_t *perm,
                          const int32_t *live, int32_t *cnt9, grpic_fields *f, bool histogram, cudaStream_t s,
                          int64_t slot0 = 0);
cudaError_t launch_deposit(grpic_ctx *ctx, const grpic_particles *b, const grpic_particles *a, const void *dphi,
                           grpic_fields *f, cudaStream_t s);
// the field update of rows [j_lo, j_hi) (j_hi < 0: every row)
cudaError_t launch_field64(grpic_ctx *ctx, grpic_fields *f, cudaStream_t s, int j_lo = 0, int j_hi = -1);
cudaError_t launch_field64_stages(grpic_ctx *ctx, double *const Xn[6], double *const J[3], double *const *Y, int64_t ld,
                                  cudaStream_t s);
cudaError_t launch_field32(grpic_ctx *ctx, grpic_fields *f, cudaStream_t s, int j_lo = 0, int j_hi = -1);
cudaError_t launch_tables_at(grpic_ctx *ctx, double a, double *tab, double *col1d, cudaStream_t s);
// the analytic initial fields (FP64) of spin a with the tables `tab` of that spin
cudaError_t launch_init_fields_at(grpic_ctx *ctx, double a, const double *tab, int kind, double B0,
                                  const grpic_fields *f, cudaStream_t s);
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int32_t *bsum, int64_t n, cudaStream_t s);
cudaError_t ensure_rad_scratch(grpic_ctx *ctx, int64_t cap);
cudaError_t launch_append_children(grpic_ctx *ctx, grpic_particles *p, cudaStream_t s);
cudaError_t launch_injection(grpic_ctx *ctx, grpic_particles *p, const grpic_fields *f, cudaStream_t s);
cudaError_t launch_keys(grpic_ctx *ctx, const grpic_particles *p, cudaStream_t s);
cudaError_t sort_setup();
cudaError_t launch_sort(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, cudaStream_t s);
// the step's sort; materialize = false leaves the order in ctx->d_perm
// (destination slot -> source slot) and the particle data where it is
// counts_ready: the push already filled d_cnt9 (neighbour path only)
cudaError_t launch_sort_step(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, bool neighbour,
                             bool hist_on_fallback, bool materialize, bool counts_ready, cudaStream_t s);
cudaError_t launch_hist(grpic_ctx *ctx, const grpic_particles *p, cudaStream_t s);
grpic_status ensure_field_scratch_ext(grpic_ctx *ctx, int64_t ld);
grpic_status ensure_particle_scratch_ext(grpic_ctx *ctx, int64_t n);
cudaError_t launch_diag(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, void *rho, void *divD,
                        cudaStream_t s);
cudaError_t launch_charge_check(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, double *rho,
                                double *divD, const double *base, double *state, unsigned long long *out,
                                cudaStream_t s);
}  // namespace grpic
