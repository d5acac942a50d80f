/*
 * grpic.h -- C ABI of the GB300 GRPIC time-step library (libgrpic.so).
 *
 * Method: Chen, Luepker & Yuan, "Introducing APERTURE: a GPU-based general
 * relativistic particle-in-cell simulation framework", arXiv:2503.04558.
 * The calls follow the paper's statement of the problem: the Kerr-Schild
 * 3+1 metric and log-r x theta Yee mesh (Sec. 2, App. A), the D/B field
 * solver (Sec. 2.1, App. B), the generalized Boris + geodesic pusher
 * (Sec. 2.2), the Esirkepov deposit (Sec. 2.3) and the step order of
 * Fig. stepping.  A particle sort by cell (not in the paper) keeps the
 * deposit coherent.
 *
 * Conventions shared by every call
 * --------------------------------
 * Units M = 1, c = 1, Heaviside-Lorentz (Sec. 2.1).  Index i runs in r,
 * j in theta.  Logical coordinates x1 = ln(r/r_in)/dx1, x2 = theta/dtheta with
 * dx1 = ln(r_out/r_in)/n_r and dtheta = pi/n_theta.  Cell key = j*n_r + i.
 *
 * Field arrays (caller-owned device memory): every component is a row-major
 * array of (n_theta+1) rows and `ld` columns (ld >= n_r + 4 and
 * (n_theta+1) * ld < 2^31, the kernels' element offsets being 32-bit), element type
 * double (precision 64) or float (precision 32).  Row j is the theta index;
 * column c = i + 2 holds the r index i of the component's own lattice
 * (Fig. Yee): D^r, B^theta, J^r at (i+1/2, j); D^theta, B^r, J^theta at
 * (i, j+1/2); D^phi, J^phi at (i, j); B^phi at (i+1/2, j+1/2).  Two guard
 * columns on each side hold the zero-derivative copies of Sec. 2.1.
 * J holds the integrated currents of the deposit, J^r A^D_r, J^theta A^D_theta
 * and J^phi dV (the quantities of Eq. J-integral-eqn with dphi = 1), which the
 * field update divides by the face areas.
 *
 * Particles (caller-owned device memory, structure of arrays):
 *   precision 64: x1 = r, x2 = theta (double), u1..u3 = covariant u_r,
 *                 u_theta, u_phi (double); `cell` unused.
 *   precision 32: cell = j*n_r + i (int32), x1, x2 = offsets in [0,1] inside
 *                 the cell in logical units (float), u1..u3 float.  In the
 *                 last theta row (j = n_theta - 1) x2 is the distance to the
 *                 pole, q = n_theta - theta/dtheta, so that theta near pi
 *                 keeps FP32's relative precision as theta near 0 does in
 *                 row 0 (x2 = theta/dtheta there); grpic_fp32_encode and
 *                 grpic_fp32_decode convert.
 *   tag: species in bits 0-1 (indexes q_over_m/q_weight/massive), bit 31 =
 *   dead.  `n` is the number of slots the call may touch; if `d_count` is not
 *   NULL it points at a device int64 holding the live count, which bounds
 *   every kernel and which grpic_sort rewrites.
 *
 * Errors: argument errors return at once.  Errors found on the device (a
 * particle moving more than one cell, a non-finite state, a wait that ran
 * out) are latched in a device status word; they surface as the return value
 * of grpic_sync() (or of the next call that synchronizes).  No call traps or
 * throws.  Every call is asynchronous on the CUDA stream passed as `stream`
 * (a cudaStream_t; NULL = the legacy default stream).
 */
#ifndef GRPIC_H
#define GRPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRPIC_OK = 0,
    GRPIC_EINVAL = 1,    /* invalid argument                                  */
    GRPIC_ENOMEM = 2,    /* device allocation failed                          */
    GRPIC_ECUDA = 3,     /* CUDA runtime error                                */
    GRPIC_ERANGE = 4,    /* a particle moved more than one cell in a step     */
    GRPIC_ENAN = 5,      /* a particle state became non-finite                */
    GRPIC_EOVERFLOW = 6, /* capacity exceeded                                 */
    GRPIC_ECONVERGE = 7, /* an iteration did not converge                     */
    GRPIC_ETIMEOUT = 8   /* a device-side wait gave up                        */
} grpic_status;

typedef struct grpic_ctx grpic_ctx;

typedef enum { GRPIC_METRIC_KERR_SCHILD = 0 } grpic_metric;

/* Analytic initial fields (App. C and Sec. 3.2). */
typedef enum {
    GRPIC_FIELD_WALD = 0,           /* rotating Wald solution, Eq. wald-solution-ks */
    GRPIC_FIELD_WALD_A0 = 1,        /* a = 0 Wald in the spinning metric, Eq. vacuum-nonrotating-wald */
    GRPIC_FIELD_MONOPOLE = 2,       /* monopole, App. C                              */
    GRPIC_FIELD_SPLIT_MONOPOLE = 3  /* sgn(cos theta) x monopole                     */
} grpic_field_kind;

/* log-r x theta mesh (Sec. 2.1): n_r x n_theta cells, r in [r_in, r_out],
 * theta in [0, pi]; outer damping layer over the last damp_cells cells with
 * factor 1 - damp_max s^3 (s = depth into the layer, 0..1). */
typedef struct {
    int32_t n_r, n_theta;
    double r_in, r_out;
    int32_t damp_cells;
    double damp_max;
} grpic_grid;

/* Solver settings.  beta_field is the semi-implicit weight beta of Eq.
 * fld-corrector (alpha = 1 - beta), n_field_iter its number of corrector
 * iterations N; n_push_iter the number of trapezoidal corrector iterations of
 * Eq. geodesic-corrector.  Per species s (tag bits 0-1): q_over_m[s] is q/m
 * in the Lorentz force, q_weight[s] the macro charge q*w deposited, massive[s]
 * the epsilon of u^0 (1 massive, 0 photon: no Boris step, Sec. 2.2).
 * precision: 64 (FP64 path) or 32 (FP32 form).  fp64_radius: in the FP32 form,
 * metric evaluations of particles in cells whose inner edge lies below
 * fp64_radius run in extended precision (<= 0: never), with the arithmetic
 * island_arith selects: 0 double-FP32 pairs (~48-bit significands on the
 * FP32 pipes, the default), 1 native FP64.  push_tol: in the FP32 form, the
 * geodesic corrector stops once the change of the iterate (r relative to r_i,
 * theta in radians, u relative to max(1, |u|)) falls below push_tol (<= 0:
 * always n_push_iter correctors).  The change is exact: two floats within a factor 2
 * subtract exactly (Sterbenz's lemma), so the test takes the FP64 decision
 * for converging iterates.  The FP64 path always runs n_push_iter.
 * pusher: the momentum update of charged particles (Sec. 2.2): 0 the
 * generalized Boris step (Eqs. boris-plus-minus .. boris-scheme, the
 * default), 1 Vay's update in the FIDO frame (the paper's alternative; the
 * differentiable form supports 0 only).
 * shape_order: the particle shape of the interpolation and of the
 * Esirkepov deposit (Sec. 2.3): 1 cloud in cell (the default), 3 the
 * third-order (cubic B-) spline, FP64 path only (the FP32 form and the
 * differentiable form refuse it).  With the cubic shape a particle's cloud
 * reaches two rows past the polar axis, folded back with the axis parities,
 * and two columns into the guard columns.
 * radiation (FP64 path, Sec. 4 on the 2D grid): after its push a charged
 * particle (species 0, 1, 2 with q != 0) whose FIDO Lorentz factor reaches
 * gamma_thr emits a photon (species 3) of FIDO energy eps_ph along its
 * momentum and keeps the rest; a photon of FIDO energy e > 2 converts with
 * probability 1 - exp(-tau dt) into an e- (species 0) and an e+ (species 1)
 * of FIDO energy e/2 each along its momentum.  injection (FP64 path, the
 * plasma-filled Wald run): after the field update every cell whose
 * magnetisation B^2 / n exceeds sigma_thr and whose |D.B| / B^2 exceeds
 * eps_db gets an e-/e+ pair at rest in the FIDO frame at a random point
 * (n: charged particles in the cell, at least one, times |q_weight[0]| over
 * the cell's volume).  Random numbers: Philox4x64-10 keyed on (seed, 0),
 * counter (slot or cell, step, event, 0).  New particles are appended after
 * the live slots in parent (cell) order, before the sort; with radiation or
 * injection grpic_step and grpic_step_graph treat the whole capacity as the
 * slot range (p->n is set to p->capacity; the device count holds the live
 * particles) and report GRPIC_EOVERFLOW when it fills. */
typedef struct {
    double dt;
    double beta_field;
    int32_t n_field_iter;
    int32_t n_push_iter;
    double q_over_m[4];
    double q_weight[4];
    int32_t massive[4];
    int32_t precision;
    int32_t sort_every;
    double fp64_radius;
    double push_tol;
    int32_t island_arith;
    int32_t pusher;
    int32_t shape_order;
    int32_t radiation;
    int32_t injection;
    double gamma_thr, eps_ph, tau;
    double sigma_thr, eps_db;
    uint64_t seed;
} grpic_params;

typedef struct {
    int64_t n;          /* slots the call may touch (upper bound of the live count) */
    int64_t capacity;   /* allocated slots of every array                          */
    int64_t *d_count;   /* optional device int64: live count (bounds kernels)      */
    void *x1, *x2;      /* r, theta (double) | in-cell offsets (float)             */
    void *u1, *u2, *u3; /* covariant u_r, u_theta, u_phi                           */
    uint32_t *tag;      /* species | dead bit                                      */
    int32_t *cell;      /* precision 32 only: cell key                             */
} grpic_particles;

typedef struct {
    void *D[3];   /* D^r, D^theta, D^phi   */
    void *B[3];   /* B^r, B^theta, B^phi   */
    void *J[3];   /* J^r A_r, J^theta A_theta, J^phi dV (deposit output) */
    int64_t ld;   /* row stride in elements, >= n_r + 4 */
} grpic_fields;

/* Create a context: validates the grid and parameters (a in [0,1),
 * 0 < r_in < r_out, n_r, n_theta >= 4 and even n_theta, dt > 0, precision 64
 * or 32), computes on the current device the face areas of Eq. area-element
 * by 10-point Gauss-Legendre quadrature and the metric coefficient products of
 * Eqs. auxE/auxH, and allocates the field-solver and sort scratch.  The
 * context owns only those tables and scratch.  *out = NULL on failure. */
grpic_status grpic_init(grpic_metric metric, double spin, const grpic_grid *grid, const grpic_params *params,
                        grpic_ctx **out);

/* Fill D and B with an analytic solution of App. C: B^r, B^theta by Stokes'
 * theorem on A_phi over each face, B^phi as the face average of the closed
 * form, D^j = gamma^{ji}(E_i - e_ikl beta^k B^l)/alpha at each D location
 * (Eq. E-H-B-D); guard cells and axis values per Sec. 2.1.  J is zeroed. */
grpic_status grpic_init_fields(grpic_ctx *ctx, grpic_field_kind kind, double B0, grpic_fields *f, void *stream);

/* Push + deposit (Sec. 2.2-2.3, Fig. stepping): for every live particle,
 * interpolate D, B at x^n, one full generalized Boris step (Eqs.
 * boris-plus-minus, u0bar, boris-scheme; skipped for photons), the geodesic
 * predictor and n_push_iter correctors (Eqs. geodesic-predictor/-corrector),
 * axis reflection, then the Esirkepov deposit of the move x^n -> x^{n+1}
 * (Eqs. esirkepov-decomp, j-phi-deposit) into f->J (zeroed first).
 * Particles that leave [r_in, r_out) are marked dead after their deposit.
 * The cell keys of the new positions are kept in the context for grpic_sort.
 * In an FP32 context each push (here and inside grpic_step, grpic_step_graph
 * and grpic_step_host) first copies D and B, on `stream`, into the context's
 * stencil quads (the four corners of each component's bilinear stencil as
 * one 16-byte element, 96 bytes per grid point, allocated with the field
 * scratch on first use), which the push's interpolation reads: changes to
 * D, B between pushes are always seen. */
grpic_status grpic_push(grpic_ctx *ctx, grpic_particles *p, grpic_fields *f, void *stream);

/* Deposit only: adds the Esirkepov currents of the moves from `before` to
 * `after` (same slots, precision-matched), with the azimuthal displacement
 * dphi[k] (device array of double or float), into f->J (not zeroed). */
grpic_status grpic_deposit(grpic_ctx *ctx, const grpic_particles *before, const grpic_particles *after,
                           const void *dphi, grpic_fields *f, void *stream);

/* Field update n -> n+1 (Eqs. fld-predictor, fld-corrector, App. B) with
 * the currents in f->J: one predictor and n_field_iter correctors, the axis
 * and inner-boundary conditions after every stage (Eq. Dr-axis for D^r on the
 * axis), the outer damping layer once at the end. */
grpic_status grpic_field_update(grpic_ctx *ctx, grpic_fields *f, void *stream);

/* How an FP32 context runs the field update: fused != 0 (the default) by
 * launches of four stages each on tiles staged in shared memory by the tensor
 * copy engine (56 x 16 points per CTA plus a halo of 4, the stages inside a
 * launch updating one point less of halo each), the result copied back into
 * f's arrays; fused = 0 one launch per stage.  Both run the same operations
 * per point (the fields agree to FP32 rounding: the compiler contracts a few
 * multiply-adds differently in the two kernels).  The fused path needs
 * 16-byte aligned arrays and ld * 4 a
 * multiple of 16 (otherwise the per-stage path runs); the row-restricted
 * update and FP64 contexts always use the per-stage path.  No device work. */
grpic_status grpic_set_field_path(grpic_ctx *ctx, int32_t fused);

/* Stable sort of the particles by cell key (dead particles last, dropped).
 * Keys are recomputed from the particle positions.  The sorted arrays are
 * written to `scratch` (same layout and capacity); on return the two structs'
 * array pointers are swapped so *p holds the sorted state.  The new live count
 * is written to p->d_count when given (p->n is left as an upper bound). */
grpic_status grpic_sort(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, void *stream);

/* nsteps full steps in the order of Fig. stepping: grpic_push (with deposit),
 * grpic_field_update, and grpic_sort every params.sort_every steps (0 = never). */
grpic_status grpic_step(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f, int nsteps,
                        void *stream);

/* The same steps as grpic_step (sort_every must be 1) replayed from a CUDA
 * graph of two steps (push, field update, sort, twice), captured on the first
 * call for these buffers and again whenever a buffer pointer or size changes.
 * When *p is not the output of the last sort one eager step runs first, so
 * that both captured sorts are neighbour sorts; an odd remainder also runs
 * eagerly.  The capture runs on a private stream and synchronizes the device
 * once; replays are enqueued on `stream`.  p and scratch are swapped as in
 * grpic_step. */
grpic_status grpic_step_graph(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, grpic_fields *f,
                              int nsteps, void *stream);

/* nsteps steps of grpic_step with the particle state resident in host
 * memory (Fig. stepping; the end-to-end form of the step).  Each step copies
 * host->n slots of the host arrays into the device buffers *dev, runs one
 * grpic_step(ctx, dev, dev_scratch, f, 1), reads the live count and copies
 * the live particles back into the same host arrays; host->n is set to the
 * live count on return.  host_f: NULL, or host arrays of D and B (J unused)
 * of f's layout, copied in before and out after every step as well.
 *   host: arrays of the precision's layout (x1, x2, u1, u2, u3, tag, and cell
 *     for precision 32) in host memory, pinned (cudaHostAlloc) for the copies
 *     to run asynchronously; host->capacity >= host->n.  d_count unused.
 *   dev, dev_scratch: device buffers as grpic_step's p and scratch
 *     (capacity >= host->n; dev->d_count required); swapped as in grpic_step.
 *   bytes: NULL or two int64 receiving the bytes copied host to device and
 *     device to host over the call.
 * The slot range is copied in chunks on two streams of the context (host to
 * device, device to host), a step's copy in of a chunk waits only for the
 * previous step's copy out of the same slots, so the directions overlap, and
 * the push runs chunk by chunk as the copies land (D and B first).
 * The host arrays are ready once `stream` has completed (the call
 * synchronizes `stream` once per step to read the live count).  Radiation
 * and injection contexts: GRPIC_EINVAL.  A failing step's status is returned
 * with the host arrays holding the last completed step. */
grpic_status grpic_step_host(grpic_ctx *ctx, grpic_particles *host, grpic_particles *dev, grpic_particles *dev_scratch,
                             const grpic_fields *host_f, grpic_fields *f, int nsteps, int64_t bytes[2],
                             void *stream);

/* Diagnostics at vertices: rho = sum q w S / dV (cloud in cell) into rho[]
 * and the discrete div D of Eq. J-integral-eqn's integral form into divD[];
 * both (n_theta+1) x ld arrays of the field precision (device). */
grpic_status grpic_diagnostics(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, void *rho, void *divD,
                               void *stream);

/* Running charge-conservation check of Sec. 3.4 (the FP32 form's FP64
 * check): rho of the particles (cloud in cell, accumulated in FP64 whatever
 * the precision) and div D (Eq. J-integral-eqn, formed in FP64 from the
 * stored D) at the vertices; out[0] = max |div D - rho - base| and out[1] =
 * max |rho| over the interior vertices (columns 1 .. n_r - damp_cells - 1, all
 * rows, from column 2 with the cubic shape; the guard copies and the damping
 * layer change div D by design), as
 * host doubles.  base: NULL or a device (n_theta+1) x ld FP64 array of an
 * earlier call's div D - rho (so that out[0] measures the change since);
 * state: NULL or such an array to receive this call's div D - rho.  p may be
 * NULL (no particles).  Synchronizes `stream`. */
grpic_status grpic_charge_check(grpic_ctx *ctx, const grpic_particles *p, const grpic_fields *f, const double *base,
                                double *state, double out[2], void *stream);

/* Copy the face areas of Eq. area-element (A^D_r, A^D_theta, A^D_phi = dV,
 * A^B_r, A^B_theta, A^B_phi) into six caller device arrays of
 * (n_theta+1) x ld doubles. */
grpic_status grpic_get_areas(grpic_ctx *ctx, double *const out[6], int64_t ld, void *stream);

/* Wait for the context's work on `stream`, read and clear the device status
 * word, and return the first device error recorded (GRPIC_OK if none). */
grpic_status grpic_sync(grpic_ctx *ctx, void *stream);

/* Phase timing of grpic_step: with enable != 0, every step of grpic_step
 * records CUDA events on its stream around the push (fused deposit), the
 * field update and the sort; enable = 0 stops it (grpic_step_graph's
 * captured steps are never timed).  grpic_get_timing waits for the recorded
 * events and writes out[0..2] = the summed milliseconds of push, field update
 * and sort over the steps since the last read or enable, and *nsteps their
 * number, then starts a new sum.  Events are created as needed (not inside a
 * capture). */
grpic_status grpic_set_timing(grpic_ctx *ctx, int enable);
grpic_status grpic_get_timing(grpic_ctx *ctx, double out[3], int64_t *nsteps);

/* ------------------------------------------------------------------------ */
/* Differentiable form (FP64 contexts only).  The objective is the time-     */
/* averaged radial Poynting flux of the 3+1 fields (S = E x H, Sec. 2.1's    */
/* auxiliary E_i, H_i of App. B) through the ring of cell faces at column    */
/* i_H (the paper defines no objective; this is the reading used here):      */
/*   flux(F) = sum_j (E_theta H_phi - E_phi H_theta)(r_{i_H}, theta_{j+1/2})  */
/*             dtheta,   with H_phi, E_phi, H_theta averaged onto that point  */
/*             from their staggered locations (2, 2 and 4 points),            */
/*   L = (1/N) sum_{n=0}^{N-1} flux(F^{n+1}),                                  */
/* where one step is grpic_push (fields n, deposit into J) followed by       */
/* grpic_field_update (no sort: it only permutes the particles).             */
/* ------------------------------------------------------------------------ */

/* flux(F) of the fields in f (D, B; J unused) into *out (host double).
 * 1 <= i_horizon <= n_r - 1.  Synchronises `stream`. */
grpic_status grpic_horizon_flux(grpic_ctx *ctx, const grpic_fields *f, int i_horizon, double *out, void *stream);

/* Transpose of one field update (Eqs. fld-predictor, fld-corrector with the
 * boundary copies and the outer damping; n_field_iter >= 1): given the
 * adjoint lam_in->D/B of the fields after the update, writes the adjoint of
 * the fields before it into lam_out->D/B and the adjoint of the integrated
 * currents J A into lam_out->J.  All arrays (n_theta+1) x ld device doubles,
 * lam_in->ld == lam_out->ld; lam_in is not modified.  Allocates and frees
 * its scratch (24 arrays); synchronises `stream`. */
grpic_status grpic_adjoint_field_step(grpic_ctx *ctx, const grpic_fields *lam_in, grpic_fields *lam_out,
                                      void *stream);

/* Forward run of nsteps steps from (p0, f0) and the reverse sweep of its
 * hand-written adjoint: particles by the transposed deposit, axis reflection,
 * the transposed geodesic step (see trapezoid_ift), the Boris Jacobian and
 * the transposed interpolation; fields by the transposed stage sequence.  The forward
 * states are recomputed from checkpoints taken every checkpoint_every steps
 * (memory: ceil(nsteps/checkpoint_every) + checkpoint_every + 2 copies of
 * the particle and field state, and the FP64 push's record of one segment:
 * checkpoint_every x (10 + 6 n_push_iter) doubles per particle).  The last
 * segment is recorded during the forward pass itself, so checkpoint_every >=
 * nsteps trades that memory for no recomputation at all.
 *   p0:  n live or dead particles (FP64 SoA r, theta, u_r, u_theta, u_phi,
 *        tag); not modified.  p0->d_count is ignored (p0->n is used).
 *   f0:  the fields at step 0 (D, B; f0->J unused); not modified.
 *   L_out: host double, the objective L.
 *   grad_p[5]: device arrays of n doubles: dL/d(r, theta, u_r, u_theta,
 *        u_phi) of every particle at step 0 (0 for dead ones).
 *   grad_f[6]: NULL or device arrays (n_theta+1) x f0->ld for dL/dD^r,
 *        dL/dD^theta, dL/dD^phi, dL/dB^r, dL/dB^theta, dL/dB^phi at step 0,
 *        entry by entry (guard columns included); a NULL entry is skipped.
 * trapezoid_ift selects the particle Jacobian of the geodesic step:
 *   0  the transpose of the predictor and the n_push_iter correctors exactly
 *      as the push runs them (the gradient of the computed trajectory);
 *   1  the implicit-function theorem at the converged trapezoid, one 5x5
 *      transposed solve per particle: the gradient of the trapezoidal rule
 *      itself, equal to 0 up to the iteration's residual (near the polar
 *      axis, where dt/2 |dF/dy| approaches 1, three correctors do not
 *      converge and the two differ).
 *   dL_da: NULL or a host double: the derivative of L with respect to the
 *        spin a at fixed step-0 state (p0, f0), fixed grid (r_in, r_out,
 *        n_r, n_theta), dt and i_horizon.  It collects the metric of every
 *        push (Boris and geodesic right-hand sides, exactly: a third dual
 *        slot in their hand-written reverse passes), the tables of every
 *        field update and of the objective (face-area inverses and metric
 *        products of App. B) contracted with the stage adjoints, the tables'
 *        a-derivatives taken by a central difference h = 1e-5 of the
 *        quadratures.  Initial fields that depend on a (the Wald solution)
 *        add sum grad_f . dF0/da: grpic_adjoint_spin adds it.  Requires grad_p;
 *        costs per step one field update more and (n_field_iter + 1) * 6 + 3
 *        field arrays of memory per checkpoint segment.
 * n_push_iter must not exceed 16 (the adjoint keeps the iterates).
 * A particle the forward refuses (ERANGE, ENAN) contributes no gradient and
 * its status is returned after the sweep.  Synchronises `stream`. */
grpic_status grpic_adjoint_grad(grpic_ctx *ctx, const grpic_particles *p0, const grpic_fields *f0, int nsteps,
                                int checkpoint_every, int i_horizon, int trapezoid_ift, double *L_out,
                                double *const grad_p[5], double *const grad_f[6], double *dL_da, void *stream);

/* dL/da of a run that starts from the analytic fields `kind`, B0 of the
 * context's spin a (App. C): runs grpic_adjoint_grad from those fields and
 * adds to its fixed-state part the step-0 fields' own dependence on a,
 * sum over every entry of dL/dF0 . dF0/da, with dF0/da the central
 * difference (h = 1e-5) of the closed-form initialization at a +- h, each
 * with the face areas of its own spin (the grid, dt and i_horizon stay those
 * of the context).  The paper defines no objective (see grpic_adjoint_grad).
 *   p0, nsteps, checkpoint_every, i_horizon, trapezoid_ift, L_out, grad_p:
 *        as for grpic_adjoint_grad (grad_p required);
 *   grad_f: NULL or six device arrays (n_theta+1) x (n_r+4) receiving
 *        dL/dF0 (otherwise kept in scratch);
 *   dL_da: host double, the total derivative.
 * Allocates and frees its scratch (three field sets, two table sets);
 * synchronizes `stream`.  GRPIC_EINVAL for an FP32 context or an unknown
 * kind; statuses of particles refused by the forward pass are returned after
 * the sweep, as by grpic_adjoint_grad. */
grpic_status grpic_adjoint_spin(grpic_ctx *ctx, const grpic_particles *p0, grpic_field_kind kind, double B0,
                                int nsteps, int checkpoint_every, int i_horizon, int trapezoid_ift, double *L_out,
                                double *const grad_p[5], double *const grad_f[6], double *dL_da, void *stream);

/* The objective's column: *out = round(ln(r_H / r_in) / dx1), the r index
 * nearest the outer horizon r_H = 1 + sqrt(1 - a_nominal^2) of the spin
 * a_nominal on the context's grid (the index is held fixed when the spin is
 * varied).  No device work. */
grpic_status grpic_horizon_index(const grpic_ctx *ctx, double a_nominal, int32_t *out);

/* ------------------------------------------------------------------------ */
/* Batched 1D spark gaps: the radiative pair-production prescription of     */
/* Sec. 4 (threshold photon emission at the FIDO Lorentz factor gamma_thr    */
/* with FIDO energy eps_ph along the emitter's momentum; photon conversion   */
/* with probability 1 - exp(-tau dt) per step, Eq. optical-depth, into an   */
/* e-/e+ pair sharing the photon's FIDO energy) on many independent radial  */
/* field lines of a monopole Kerr magnetosphere.  Each line k at fixed      */
/* theta_k has n_cells cells uniform in ln r on [r_in, r_out] and one field */
/* component D^r at (i+1/2) obeying d(A_r D^r)/dt = I0_k - J^r A_r (A_r =    */
/* sqrt(gamma) at (r_{i+1/2}, theta_k), I0_k an imposed line current).      */
/* Particles slide along the line (theta frozen, u_theta = 0, u_phi kept):  */
/* electric kick q/m alpha dt gamma_rr D^r, geodesic predictor-corrector in */
/* (r, u_r) (Eqs. geodesic-predictor/-corrector), 1D Esirkepov deposit.      */
/* Random draws: Philox4x64-10 keyed on (seed, 0) with counter (particle id,*/
/* step, 1, 0); a uniform is the top 53 bits of the first output word.      */
/* Children get the id splitmix64(splitmix64(parent) ^ (step << 2 | k)),    */
/* k = 0 photon, 1 electron, 2 positron.  After each step a line holds its  */
/* surviving particles in their previous order followed by the particles    */
/* created in that step in the order of their parents.                      */
/* FP32 particles and fields; the emission threshold and the conversion     */
/* decision are taken in FP64.                                              */
/* ------------------------------------------------------------------------ */
typedef struct grpic_batch1d_ctx grpic_batch1d_ctx;

typedef struct {
    int32_t n_lines, n_cells;
    double a, r_in, r_out, dt;
    int32_t n_push_iter;
    double q_over_m[4], q_weight[4];
    int32_t massive[4];
    double gamma_thr, eps_ph, tau;
    double B0;          /* monopole strength of the initial D^r (App. C) */
    uint64_t seed;      /* Philox key word 0                              */
    int64_t capacity;   /* particle slots per line in each buffer         */
} grpic_batch1d_params;

/* Caller-owned device arrays.  Line k's particles occupy slots
 * [k*capacity, k*capacity + count[k]) of buffer `cur`; the other buffer is
 * the destination of the next step (the two are swapped every step). */
typedef struct {
    double *theta;       /* [n_lines] line inclination theta_k              */
    double *I0;          /* [n_lines] imposed line current (J A units)      */
    float *D;            /* [n_lines][n_cells] D^r at i+1/2                 */
    float *JA;           /* [n_lines][n_cells+2] J^r A_r of the last step at
                            faces -1..n_cells (output; NULL = not written)  */
    int32_t *count;      /* [n_lines] particles per line                    */
    int32_t *cell[2];    /* cell index i along the line                     */
    float *off[2];       /* offset in [0,1) inside the cell (logical units) */
    float *ur[2], *up[2];/* covariant u_r, u_phi                            */
    uint32_t *tag[2];    /* species 0 e-, 1 e+, 3 photon (| bit 31 dead)    */
    uint64_t *id[2];     /* particle identity (RNG counter)                 */
    int32_t cur;         /* buffer holding the state; updated by the runs   */
    unsigned long long *events; /* [3] accumulated photons emitted, photons
                                   converted, particle pushes performed     */
} grpic_lines;

/* Validate the parameters, build the radius table and the staging scratch
 * (appended particles of one step, capacity/2 slots per line). */
grpic_status grpic_batch1d_init(const grpic_batch1d_params *params, grpic_batch1d_ctx **out);

/* A_r along every line and the initial D^r of the monopole (App. C) at
 * (r_{i+1/2}, theta_k). */
grpic_status grpic_batch1d_init_fields(grpic_batch1d_ctx *ctx, grpic_lines *lines, void *stream);

/* nsteps steps (global step numbers step0 .. step0+nsteps-1) of every line
 * in one persistent launch: CTAs take lines from a device queue ordered by
 * decreasing particle count, keep D^r and J^r A_r of their line in shared
 * memory and run all nsteps for it.  J^r A_r is summed in 64-bit fixed point
 * (units of 2^-32 |q w|_max / dt), so the current does not depend on the
 * order of the deposits and repeated runs give the same D^r bit for bit.  Capacity overflow drops the excess
 * appended particles and latches GRPIC_EOVERFLOW (read by
 * grpic_batch1d_sync). */
grpic_status grpic_batch1d_run(grpic_batch1d_ctx *ctx, grpic_lines *lines, int nsteps, int64_t step0, void *stream);

/* The same run as grpic_batch1d_run from a CUDA graph (the line-order
 * kernel, then the persistent kernel), built on the first call for these
 * line buffers and launch shape; later calls only update the persistent
 * kernel's arguments (steps, first step, current buffer) in the graph. */
grpic_status grpic_batch1d_run_graph(grpic_batch1d_ctx *ctx, grpic_lines *lines, int nsteps, int64_t step0,
                                     void *stream);

/* Autotuner: runs trial_steps real steps (starting at step0) with each
 * candidate launch shape (threads per CTA, CTAs per SM, CTAs per line),
 * times them with CUDA events and keeps the fastest for later runs.
 * Advances the state by trial_steps * (number of candidates) steps, returned
 * in *steps_done; best[0] = threads per CTA, best[1] = CTAs per SM,
 * best[2] = CTAs per line (1, or 2 as a thread-block cluster on two SMs that
 * share the line: each pushes half of its particles, the two currents are
 * summed through distributed shared memory in a fixed order, the line's
 * particle order is the same as with one CTA). */
grpic_status grpic_batch1d_tune(grpic_batch1d_ctx *ctx, grpic_lines *lines, int trial_steps, int64_t step0,
                                int64_t *steps_done, int32_t best[3], void *stream);

/* Set the launch shape of later runs (as the tuner would): threads per CTA
 * (a multiple of 32 in [32, 1024]), CTAs per SM (at most what the CTA's
 * registers and shared memory allow), CTAs per line (1 or 2).  GRPIC_EINVAL
 * for a shape that cannot run.  No device work. */
grpic_status grpic_batch1d_set_launch(grpic_batch1d_ctx *ctx, int32_t threads, int32_t ctas_per_sm,
                                      int32_t ctas_per_line);

/* Wait for `stream`, return and clear the first latched device error. */
grpic_status grpic_batch1d_sync(grpic_batch1d_ctx *ctx, void *stream);

void grpic_batch1d_destroy(grpic_batch1d_ctx *ctx);

/* Largest sizes grpic_sort_noalloc accepts (the size of its fixed scratch). */
#define GRPIC_NOALLOC_MAX_PARTICLES 2097152 /* slots p->n                  */
#define GRPIC_NOALLOC_MAX_CELLS 262144      /* n_r * n_theta (e.g. 512^2)   */

/* Sort by cell without any device allocation.  The paper has no counterpart:
 * this entry exists for callers that cannot call cudaMalloc -- code running
 * while a stream is being captured, hosts whose memory pools own all device
 * memory, plugin hosts that forbid library allocations.  It computes the same
 * stable order as grpic_sort (same kernels, same result) but needs no context:
 * the grid, the precision (64 or 32) and the two particle buffers are given
 * directly, and the scratch (keys, histogram, offsets, index list) is one
 * fixed __device__ array of about 20 MB in libgrpic that every GPU loading
 * the library holds until the process exits.
 *   - The caller passes inputs and outputs as for grpic_sort: the sorted state
 *     is written into `scratch` and the two structs' array pointers are
 *     swapped on return; the live count goes to p->d_count when given.
 *   - Sizes above GRPIC_NOALLOC_MAX_PARTICLES particles or
 *     GRPIC_NOALLOC_MAX_CELLS cells return GRPIC_EOVERFLOW before any launch.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 *     first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and sets a kernel
 *     attribute; make that first call before any stream capture begins.  The
 *     look-up is kept per CUDA context: after cudaDeviceReset, or with another
 *     context current, the next call repeats it (again before any capture).
 *   - Every call shares the one array, which keeps the last call's contents
 *     (each call clears what must start at zero).  Calls that overlap on the
 *     GPU -- on different streams, or from different host threads -- race on
 *     it and corrupt each other's results: serialize them. */
grpic_status grpic_sort_noalloc(const grpic_grid *grid, int32_t precision, grpic_particles *p,
                                grpic_particles *scratch, void *stream);

/* ------------------------------------------------------------------------ */
/* theta-slab domain decomposition (the paper's multi-GPU design, Sec. 1:  */
/* the domain split among GPUs with MPI exchanges of the boundary data).    */
/* Each rank keeps field arrays of the whole grid (global row indices) but  */
/* updates only rows [j0 - G, j1 + G) around its own rows [j0, j1), and     */
/* pushes only the particles of its rows.  One step (the host driver moves  */
/* the buffers between ranks):                                              */
/*   grpic_push (own particles, J zeroed and deposited);                    */
/*   J halo reduction: the rows outside [j0, j1) that the deposit reached  */
/*   go to their owners (grpic_halo_pack / grpic_halo_unpack with add);     */
/*   then the owners' complete rows fill the G ghost rows on each side      */
/*   (pack, unpack with copy);                                              */
/*   grpic_field_update_rows on [j0 - G, j1 + G): a stage's D rows read   */
/*   the B rows at and below them and its B rows the D rows at and above    */
/*   them, so a wrong row outside the range moves half a row inwards per    */
/*   stage; with G = ceil((N + 1) / 2) for the 1 + N stages the own rows    */
/*   come out as in the undivided grid; the ghost rows of D, B are then     */
/*   refilled from their owners;                                            */
/*   migration: grpic_sort_split sorts the particles by cell and returns   */
/*   how many left below j0 and above j1 (at most one row in a step), the   */
/*   leavers are packed (grpic_particles_pack) and sent, and               */
/*   grpic_slab_assemble places [arrivals from below | own | arrivals from  */
/*   above] before a last grpic_sort; since each neighbour's order is the   */
/*   undivided run's order of its particles and a stable sort keeps the     */
/*   order of equal keys, the result is the undivided run's order of this   */
/*   slab's particles.                                                      */
/* Field sets: 0 = D^r, D^theta, D^phi, B^r, B^theta, B^phi; 1 = the three  */
/* J arrays.  A packed halo holds the components one after the other, each  */
/* as its rows [row0, row0 + nrows) exactly as in the field arrays          */
/* (nrows * ld elements of the field precision per component).  A packed    */
/* particle message of n particles holds the arrays x1, x2, u1, u2, u3 (8   */
/* or 4 bytes each), tag (4 bytes) and, in the FP32 form, cell (4 bytes),   */
/* n entries each, back to back.  Device buffers, caller-owned.             */
/* ------------------------------------------------------------------------ */

/* The field update of grpic_field_update restricted to rows [j_lo, j_hi) of
 * every component (0 <= j_lo < j_hi <= n_theta + 1); rows outside are left
 * unchanged and are read by the range's edge rows.  The axis conditions
 * apply to rows 0 and n_theta when they lie in the range. */
grpic_status grpic_field_update_rows(grpic_ctx *ctx, grpic_fields *f, int32_t j_lo, int32_t j_hi, void *stream);

/* Copy rows [row0, row0 + nrows) of field set `set` into buf (device,
 * ncomp * nrows * ld elements), or back: unpack with add = 0 copies, with
 * add != 0 adds buf to the rows (the current halo reduction). */
grpic_status grpic_halo_pack(grpic_ctx *ctx, const grpic_fields *f, int32_t set, int32_t row0, int32_t nrows,
                             void *buf, void *stream);
grpic_status grpic_halo_unpack(grpic_ctx *ctx, grpic_fields *f, int32_t set, int32_t row0, int32_t nrows,
                               const void *buf, int32_t add, void *stream);

/* grpic_sort (always the general counting sort, keys recomputed from the
 * positions) followed by the segment counts of the sorted live particles:
 * counts[0] in rows below j_lo, counts[1] in rows [j_lo, j_hi), counts[2]
 * in rows j_hi and above (0 <= j_lo <= j_hi <= n_theta), as host int64.
 * Synchronizes `stream`. */
grpic_status grpic_sort_split(grpic_ctx *ctx, grpic_particles *p, grpic_particles *scratch, int32_t j_lo,
                              int32_t j_hi, int64_t counts[3], void *stream);

/* Pack slots [first, first + n) of p into buf (the message layout above). */
grpic_status grpic_particles_pack(grpic_ctx *ctx, const grpic_particles *p, int64_t first, int64_t n, void *buf,
                                  void *stream);

/* dst slots [0, n_lower) <- the packed message `lower`, then slots
 * [own_first, own_first + own_n) of src, then the packed message `upper`;
 * dst->n is set to the total and written to dst->d_count when given (that
 * copy synchronizes `stream`).  The sort's cached keys are dropped, so the
 * next sort recomputes them. */
grpic_status grpic_slab_assemble(grpic_ctx *ctx, grpic_particles *dst, const grpic_particles *src, int64_t own_first,
                                 int64_t own_n, const void *lower, int64_t n_lower, const void *upper,
                                 int64_t n_upper, void *stream);

/* Measured arithmetic ceiling of the current device (measurement support for
 * the ALU rooflines; the paper has no counterpart).  kind 0: FP32 fused
 * multiply-add, 1: FP64 fused multiply-add, 2: packed FP32 fused multiply-add
 * (one instruction on a float pair).  Runs one full-occupancy launch of
 * independent FMA chains six times on `stream` (the first as warm-up) and
 * writes out[0] = the best rate in flop/s (2 per FMA), out[1] = the same in
 * FMA warp-instructions/s, out[2] = the SM count.  Allocates and frees an
 * 8-byte result; synchronizes `stream`. */
grpic_status grpic_alu_peak(int32_t kind, double out[3], void *stream);

/* Conversion between FP64 positions (r, theta) and the FP32 form's cell key
 * and offsets (the layout above, the last row's offset measured from the
 * pole), on the context's grid, in FP64 on the device: slots [0, n) of the
 * given device arrays.  Encoding clamps the cell to the grid. */
grpic_status grpic_fp32_encode(grpic_ctx *ctx, int64_t n, const double *r, const double *theta, int32_t *cell,
                               float *o1, float *o2, void *stream);
grpic_status grpic_fp32_decode(grpic_ctx *ctx, int64_t n, const int32_t *cell, const float *o1, const float *o2,
                               double *r, double *theta, void *stream);

/* Human-readable description of the last error seen by the context. */
const char *grpic_last_error(const grpic_ctx *ctx);

/* Free the context's tables and scratch (never the caller's buffers). */
void grpic_destroy(grpic_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRPIC_H */
