/*
 * vofl.h -- C ABI of the GB300 (sm_103a) variable-order fractional Laplacian
 * wave solver, after arXiv 2311.13049 ("Fourier pseudospectral methods for the
 * variable-order space fractional wave equations").
 *
 * What it computes
 *   The seismic viscoacoustic model of Eq. (1.1),
 *       u_tt / c^2 = eta (-Delta)^{1+gamma(x)} u + tau d/dt[(-Delta)^{1/2+gamma(x)} u],
 *   with c = c0 cos(pi gamma/2), eta = -c0^{2 gamma} w0^{-2 gamma} cos(pi gamma),
 *   tau = -c0^{2 gamma - 1} w0^{-2 gamma} sin(pi gamma), gamma = arctan(1/Q)/pi
 *   (Sec. 1), on a periodic grid (Sec. 2, Sec. 2.3).  Each variable-order
 *   operator is applied with the accelerated matrix-free scheme of Eq. (2.13):
 *       (-Delta)^{s(x_j)} u_j ~= sum_{m=0}^{M} [s(x_j)-s0]^m
 *              sum_{k != 0} (ln|mu_k|^2)^m / m! |mu_k|^{2 s0} u_hat_k e^{i mu_k.(x_j-a)},
 *   s0 = grid mean of s.  Time stepping is the leap-frog (LFFP) scheme of
 *   Eq. (3.4) extended to Eq. (1.1) (damping term by a backward difference).
 *
 * Conventions (all entry points)
 *   - Every function returns a vofl_status (0 = success, < 0 = error); none
 *     aborts or throws.  vofl_last_error() gives a message for the last error
 *     on a context.
 *   - Arrays are dense, C order, indexed [z][y][x] (x fastest); grid sizes
 *     n[] and box bounds lo[], hi[] are given in (x, y, z) order.
 *   - Grid sizes must be even (Sec. 2: "J even").  The fused kernels
 *     (VOFL_IMPL_FUSED) cover 1D lines of 16..4096 points (float; double up
 *     to 2048), the 2D grids 64^2, 128^2, 256^2, 512^2, 768^2, 1024^2,
 *     256x128, 128x256, 512x64, 64x512 and 1024x256 in float, and the 3D
 *     grids 64^3, 128^3, 256^3 and 128x64x256 in float; other shapes run on
 *     the plain cuFFT path (VOFL_IMPL_PLAIN) or return VOFL_EUNSUPPORTED.
 *   - "_dev" pointers are device pointers on the GPU current when the context
 *     was created; others are host pointers unless an `on_device` flag says so.
 *     Inputs are copied in (the caller keeps ownership); outputs go to caller
 *     buffers.  Element type follows the context precision (float for
 *     VOFL_F32, double for VOFL_F64) except where a prototype says double.
 *   - Work is queued on the context's CUDA stream and is asynchronous unless
 *     stated; errors of queued work are sticky and reported by vofl_sync().
 *   - A context is not thread-safe; distinct contexts may be used concurrently.
 */
#ifndef VOFL_H
#define VOFL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VOFL_API __attribute__((visibility("default")))
#else
#define VOFL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vofl_ctx vofl_ctx;

typedef enum {
  VOFL_OK = 0,
  VOFL_EINVAL = -1,        /* bad argument */
  VOFL_ENOMEM = -2,        /* device allocation failed */
  VOFL_ECUDA = -3,         /* a CUDA / cuFFT call failed */
  VOFL_ETIMEDOUT = -4,     /* a bounded device wait gave up */
  VOFL_ESTATE = -5,        /* call out of order (e.g. step before set_q) */
  VOFL_EUNSUPPORTED = -6,  /* size / dimension / precision not built */
  VOFL_ENOCONV = -7        /* the implicit (Crank-Nicolson) solve did not converge */
} vofl_status;

typedef enum { VOFL_F32 = 0, VOFL_F64 = 1 } vofl_prec;

/* The two operators of Eq. (1.1). */
typedef enum {
  VOFL_OP_1PG = 0, /* (-Delta)^{1+gamma(x)}   */
  VOFL_OP_HPG = 1, /* (-Delta)^{1/2+gamma(x)} */
  VOFL_OP_S = 2    /* (-Delta)^{s(x)} of the general model (vofl_set_order) */
} vofl_op;

/* Time stepping of vofl_step: the leap-frog scheme (Eq. (3.4); both
 * models), the second-order time splitting of Sec. 3.3 (general model;
 * plain path, or the fused FP32 2D path) or the Crank-Nicolson scheme of
 * Sec. 3.1 (general model, plain path). */
typedef enum {
  VOFL_SCHEME_LFFP = 0,
  VOFL_SCHEME_TSFP2 = 1,
  VOFL_SCHEME_CNFP = 2
} vofl_scheme;

/* Implementation of the operator/step: the fused hand-written kernels, or
 * the plain baseline (cuFFT transforms + separate multiply / accumulate /
 * update kernels, same arithmetic). */
typedef enum { VOFL_IMPL_FUSED = 0, VOFL_IMPL_PLAIN = 1 } vofl_impl;

/* Create a context for a periodic box prod_m [lo_m, hi_m) with n_m points
 * per axis (Sec. 2.3: x_j = a + j h, h = (b-a)/J).  ndim in {1,2,3}.
 * prec: VOFL_F32 or VOFL_F64 arithmetic for transforms and updates (the
 * per-model coefficients are always computed in double).  stream: a
 * cudaStream_t, or NULL for a stream the context creates itself (a blocking
 * stream, hence ordered with the legacy default stream).  On success *out
 * owns all device state; free it with vofl_destroy. */
VOFL_API int vofl_create(vofl_ctx** out, int ndim, const int64_t* n, const double* lo,
                         const double* hi, int prec, int impl, void* stream);
VOFL_API void vofl_destroy(vofl_ctx* ctx);

/* Quality-factor model (Sec. 1): gamma = arctan(1/Q)/pi, then c, eta, tau
 * with scalar c0, omega0.  Q has prod(n) doubles, host or device; all Q > 0.
 * Derives, in double on the GPU: gamma0 = grid mean of gamma (the s0 of
 * Eq. (2.13) for both operators, s0 = 1+gamma0 and 1/2+gamma0),
 * delta = gamma - gamma0, A = c^2 eta, B = c^2 tau, and the spectral tables
 * |mu_k|^{2 s0}, ln|mu_k|^2.  Resets the time stepper. */
VOFL_API int vofl_set_q(vofl_ctx* ctx, const double* Q, int on_device, double c0,
               double omega0);

/* General variable-order model (Sec. 1, Eq. (1.5)):
 *   u_tt = -kappa (-Delta)^{s(x)} u + f(u),  f(u) = f1 u + f3 u^3,
 * with the same matrix-free operator (Eq. (2.13), centre s0 = grid mean of
 * s, delta = s - s0) and the leap-frog scheme of Eq. (3.4a-c) (start step
 * u^1 = u^0 + dt psi + dt^2/2 (-kappa L u^0 + f(u^0))).  s: N doubles in
 * (0, 2] (host or device by on_device); kappa > 0; a point source
 * (vofl_set_source) is added as for the seismic model.  After this call
 * vofl_apply takes VOFL_OP_S (and rejects the seismic operators); a later
 * vofl_set_q / vofl_set_gamma switches back.  Resets the run.  Returns
 * VOFL_OK, VOFL_EINVAL (bad arguments or s outside (0, 2]) or VOFL_ECUDA. */
VOFL_API int vofl_set_order(vofl_ctx* ctx, const double* s, int on_device, double kappa, double f1, double f3);

/* As vofl_set_q with gamma given directly (gamma = 0 allowed: the classical
 * acoustic wave equation, Sec. 1).  c0_field (prod(n) doubles or NULL) lets
 * c0 vary in space as in the paper's two-layer example (Sec. 4.3, Example 3);
 * when NULL the scalar c0 is used. */
VOFL_API int vofl_set_gamma(vofl_ctx* ctx, const double* gamma, const double* c0_field,
                   int on_device, double c0, double omega0);

/* Select the time-stepping scheme of vofl_step (vofl_scheme).  The time
 * splitting (Sec. 3.3) integrates u_t = v, v_t = -kappa (-Delta)^{s0} u
 * exactly in Fourier space over dt/2, kicks v by
 * dt (-kappa [(-Delta)^{s(x)} - (-Delta)^{s0}] u + f(u)) (the terms
 * m = 1..M of Eq. (2.13)), and repeats the half rotation; the state is
 * (u, v) with v^0 = the v0 of vofl_set_state, and no point source is
 * applied.  It needs the general model (vofl_set_order) and the plain
 * path (VOFL_IMPL_PLAIN) or a fused FP32 2D context, else vofl_step
 * returns VOFL_EUNSUPPORTED.  On the fused 2D path the rotations run on
 * its own line transforms in FP32 and the m >= 1 terms on the operator
 * kernels (one operator, Taylor groups of the transform schedule), and
 * the two half-step rotations that meet between consecutive steps of one
 * call are one rotation over dt (the call's first and last rotations over
 * dt/2 and -dt/2 bracket them): the same scheme, one rotation per step.
 * The Crank-Nicolson scheme (Sec. 3.1, Eq. (3.2)) takes the explicit start
 * step of Eq. (3.3) (that of the leap-frog scheme), then for n >= 1 solves
 *     u^{n+1} + c L u^{n+1} - h f(u^{n+1})
 *         = 2 u^n - u^{n-1} - c L u^{n-1} + h f(u^{n-1})  (+ source),
 * c = kappa dt^2/2, h = dt^2/2, L the operator of Eq. (2.13), by a
 * fixed-point iteration on f around conjugate gradients on the normal
 * equations of A = I + c L (A is not symmetric when s varies), to the
 * tolerance of vofl_set_solver.  It needs the general model and the plain
 * path, and takes no point source (vofl_step returns VOFL_EUNSUPPORTED while one is set).
 * Returns VOFL_OK, VOFL_EINVAL (unknown scheme) or VOFL_ESTATE (a run is
 * in progress: set the state first). */
VOFL_API int vofl_set_scheme(vofl_ctx* ctx, int scheme);

/* Stopping rule of the Crank-Nicolson solve (VOFL_SCHEME_CNFP): each step
 * ends when the residual r = b + h f(v) - A v of its nonlinear system
 * (notation of vofl_set_scheme) has |r|_2 <= tol |b + h f(v)|_2; every
 * linear solve of the fixed-point iteration stops at half that residual
 * or after max_iter conjugate-gradient iterations (then vofl_step returns
 * VOFL_ENOCONV, as it does when a fixed-point pass no longer lowers a
 * residual above 10 tol: tol below what the precision reaches for this
 * step; one that stalls within 10 tol ends the step).  The k = 0 mode of
 * the scheme accumulates each step's solve error, so long FP64 runs want
 * tol near the rounding floor.  Defaults: tol = 1e-15 (VOFL_F64) or 1e-6
 * (VOFL_F32),
 * max_iter = 5000.  Returns VOFL_OK or VOFL_EINVAL (tol outside (0, 1) or
 * max_iter < 1). */
VOFL_API int vofl_set_solver(vofl_ctx* ctx, double tol, int max_iter);

/* Totals of the Crank-Nicolson solver since the state was set: conjugate-
 * gradient iterations and linear solves (fixed-point passes).  Either
 * pointer may be NULL.  Read after vofl_sync for the final values.
 * Returns VOFL_OK or VOFL_EINVAL. */
VOFL_API int vofl_solver_stats(vofl_ctx* ctx, int64_t* iterations, int64_t* solves);

/* Highest Taylor power M of Eq. (2.13): each operator apply runs the M+1
 * terms m = 0..M.  0 <= M <= 40.  Default 8. */
VOFL_API int vofl_set_M(vofl_ctx* ctx, int M);

/* out_dev = (-Delta)_h^{s(x)} u_dev for op (Eq. (2.13)): s = 1+gamma or
 * 1/2+gamma for the seismic model, s(x) of vofl_set_order for VOFL_OP_S.
 * u_dev, out_dev: device arrays of prod(n) elements of the context
 * precision; they may not alias the context's state.  Async.  VOFL_EINVAL
 * for an operator that does not belong to the model set. */
VOFL_API int vofl_apply(vofl_ctx* ctx, int op, const void* u_dev, void* out_dev);

/* Both operators of the seismic model on the same input (one forward
 * transform, both sums).  VOFL_EINVAL for the general model, whose one
 * operator is VOFL_OP_S of vofl_apply. */
VOFL_API int vofl_apply_pair(vofl_ctx* ctx, const void* u_dev, void* out1_dev,
                    void* out2_dev);

/* Initial state u(x,0) = phi, u_t(x,0) = psi (Eq. (3.4b-c) start data);
 * psi may be NULL (zero).  Arrays of the context precision, host or device.
 * Resets the step counter. */
VOFL_API int vofl_set_state(vofl_ctx* ctx, const void* u0, const void* v0,
                   int on_device);

/* Point source: adds r_n / h^d at grid index idx (x,y,z order) to the right
 * hand side of Eq. (1.1) at t_n = n dt, where r_n = samples[n] (double) for
 * n < nsamples and 0 afterwards; n counts from the start of the run.
 * nsamples = 0 removes the source.  Host or device samples. */
VOFL_API int vofl_set_source(vofl_ctx* ctx, const int64_t* idx, const double* samples,
                    int64_t nsamples, int on_device);

/* Advance nsteps leap-frog steps of size dt (Eq. (3.4a) for Eq. (1.1)):
 *   u^{n+1} = 2u^n - u^{n-1} + dt^2 [A L1 u^n + B (L2 u^n - L2 u^{n-1})/dt + f_n],
 * the first step of a run being the Taylor start
 *   u^1 = u^0 + dt psi + dt^2/2 [A L1 u^0 + B L2 psi + f_0]   (Eq. (3.4c)).
 * dt must stay the same for the whole run.  Async (steps are replayed from
 * a captured CUDA graph when the path allows it). */
VOFL_API int vofl_step(vofl_ctx* ctx, int64_t nsteps, double dt);

/* Checkpoint of a run (host memory): the grid, M, the scheme and model
 * scalars, the step count, dt, the state fields (u^n, u^{n-1} or v,
 * L2 u^{n-1}), the model fields (delta, A, B and the gamma or s field) and
 * the source samples.  With blob == NULL, *nbytes receives the size;
 * otherwise *nbytes is the buffer size on entry and the bytes written on
 * return.  Waits for the queued work.  Returns VOFL_OK, VOFL_EINVAL (null
 * nbytes, buffer too small: *nbytes then holds the size), VOFL_ESTATE (no
 * model or state) or VOFL_ECUDA. */
VOFL_API int vofl_save_state(vofl_ctx* ctx, void* blob, size_t* nbytes);

/* Resume a run from a checkpoint of vofl_save_state, into a context of the
 * same grid, box and precision (any context: the model is restored with the
 * run).  The engine's spectral tables are rebuilt from the restored model,
 * so the next steps equal those of the saved run on the same path and GPU,
 * bit for bit.  The solver counters of vofl_solver_stats restart at 0.
 * Waits for the queued work.  Returns VOFL_OK, VOFL_EINVAL (not a
 * checkpoint, another grid or precision, a size that does not match) or
 * VOFL_ECUDA. */
VOFL_API int vofl_load_state(vofl_ctx* ctx, const void* blob, size_t nbytes);

/* Copy the current wavefield u^n (n = steps taken) to u_out (host or device,
 * context precision).  Synchronises the stream when the target is host
 * memory. */
VOFL_API int vofl_get_state(vofl_ctx* ctx, void* u_out, int on_device);

/* Non-blocking completion check: 1 if every piece of work queued on the
 * context's stream has finished, 0 if some is still running, < 0 on a CUDA
 * error.  Works on a context held by a batch (its stream then also waits
 * for the batch's work queued before vofl_batch_remove). */
VOFL_API int vofl_query(vofl_ctx* ctx);

/* Time step for a run of the current model: dt = courant * 2 / omega_max,
 * omega_max = max_x |c^2 eta|^{1/2} |mu_max|^{1+gamma(x)} with |mu_max| the
 * largest grid wavenumber (sqrt of the sum of (pi n_i / L_i)^2): the
 * highest angular frequency of the undamped part of Eq. (1.1) on the grid,
 * against which explicit leap-frog needs dt < 2 / omega.  courant = 0.25 is
 * the rule the built-in workloads use.  Blocks until done.  Returns VOFL_OK,
 * VOFL_EINVAL, VOFL_ESTATE (no model) or VOFL_ECUDA. */
VOFL_API int vofl_suggest_dt(vofl_ctx* ctx, double courant, double* dt);

/* Taylor power for a truncation tolerance (Sec. 2.2, the choice of M):
 * the smallest M in [0, 40] with a^{M+1}/(M+1)! e^{2a} <= tol, where
 * a = max_x |s(x) - s0| * max_k |ln |mu_k|^2| (k != 0): every mode's weight
 * |mu_k|^{2 s0} exp((s(x) - s0) ln|mu_k|^2) of Eq. (2.13) is then
 * reproduced to relative error tol by the terms m = 0..M (Taylor
 * remainder).  *M receives it (40 if none suffices); the context's M is not
 * changed (vofl_set_M).  Blocks until done.  Returns VOFL_OK, VOFL_EINVAL,
 * VOFL_ESTATE (no model) or VOFL_ECUDA. */
VOFL_API int vofl_suggest_M(vofl_ctx* ctx, double tol, int* M);

/* Number of steps taken in the current run. */
VOFL_API int64_t vofl_steps_taken(const vofl_ctx* ctx);

/* Wait for queued work; returns the first sticky error of that work. */
VOFL_API int vofl_sync(vofl_ctx* ctx);

VOFL_API const char* vofl_last_error(const vofl_ctx* ctx);

/* Device bytes a context of this shape needs (for admission by footprint). */
VOFL_API size_t vofl_footprint_bytes(int ndim, const int64_t* n, int prec, int impl,
                            int M);

/* Number of kernels this library has launched in the calling process
 * (counted at the launch sites; a captured graph counts its kernels each
 * time it is replayed). */
VOFL_API uint64_t vofl_kernel_launches(void);

/* Time each kernel kind of one fused step in isolation (CUDA events on the
 * context stream, reps launches each, after one warm-up).  names_out gets a
 * ';'-separated list of kernel names (cap bytes), ms_out (cap entries) the
 * average milliseconds per launch, units_out the lines (1D transforms)
 * each launch processes.  Returns the number of entries written, or < 0. */
VOFL_API int vofl_profile_kernels(vofl_ctx* ctx, int reps, char* names_out,
                         size_t names_cap, double* ms_out,
                         double* units_out, int cap);

/* Accuracy diagnostics (the relative L2 measure in which every result of
 * this library is stated): with x, y two fields of the context's grid
 * (N = prod(n) elements each, device pointers on the context's device,
 * element type float for VOFL_F32, double for VOFL_F64, chosen per
 * argument), on the GPU with FP64 accumulation and a fixed reduction order:
 *   out[0] = ||x - y||_2 / ||y||_2,   out[1] = max|x - y| / max|y|,
 *   out[2] = ||y||_2,                 out[3] = max|y|
 * (a ratio is 0 when x = y = 0 and +inf when only y is zero; the ratios
 * and the maxima are NaN when either field holds a NaN).  Runs on the
 * context stream after its queued work and waits for the result.  Uses the
 * context's reduction scratch; needs no model or state.  Returns VOFL_OK,
 * VOFL_EINVAL or VOFL_ECUDA. */
VOFL_API int vofl_rel_l2(vofl_ctx* ctx, const void* x_dev, int x_prec, const void* y_dev, int y_prec,
                         double* out);

/* Transform schedule of the fused 2D path.  The paper has no counterpart:
 * it fixes how the same arithmetic of Eq. (2.13) is laid out on the GPU,
 * not what is computed.  Results of different schedules agree within the
 * FP32 tolerance but not bit for bit (the multiplier recurrence restarts at
 * other terms, lines are transformed with other radices).
 *   wide_cols, wide_rows: 1 = the inverse column / row pass transforms its
 *     512- or 1024-point lines with 16 elements per lane over N/16 lanes
 *     (three radix stages, two warps per 1024-point line), 0 = with up to
 *     32 elements per lane over one warp (two stages), -1 = the size's
 *     default (wide columns at 512, wide rows at 512 and 1024); ignored
 *     (reported 0) for other line lengths.
 *   col_parts: runs of terms per Taylor group in the inverse column pass
 *     (each run starts its multiplier recurrence afresh), 1..41, or 0 for
 *     the size's default (3 at ny <= 256, 6 at ny <= 512, 1 above); not
 *     used while col_pack > 0.
 *   group: Taylor terms per group G (the terms whose per-term column
 *     transforms are stored between the column and row passes), 1..41;
 *     0 = the default, 17 (M <= 16 in one group).  Changing it re-sizes
 *     that buffer (a device allocation).
 *   fuse_forward: 1 = the top group's inverse column kernel also does the
 *     forward transform along y (one launch fewer per step; the same
 *     arithmetic, so the same bits), 2 = both forward passes (32-element
 *     lines) in one cooperative launch with a grid-wide barrier between
 *     them (the same bits as the two kernels; not with wide_fwd = 1),
 *     0 = separate forward row and column kernels, -1 = the default (1 on
 *     grids of up to 256 rows, 2 on square grids of 512, 768 and 1024);
 *     reported 0 when the column pass is wide (1), or when the forward
 *     rows are wide or the device cannot launch it (2).
 *   wide_fwd: 1 = the forward row pass transforms its 512- or 1024-point
 *     lines with the wide line transform (as wide_rows), 0 = 32 elements
 *     per lane, -1 = the default (0); reported 0 for other line lengths.
 *   row_split: runs of terms each row's group is split into in the
 *     32-element row pass, one warp per run, the runs' Horner sums joined
 *     by Horner's rule (1, 2 or 4, dividing that kernel's warps per CTA; 0
 *     = the default: 4 up to 256^2 points, else 1); reported 1 when the row
 *     pass is wide.
 *   col_pack: K > 0 (up to 65535) = the inverse column pass runs on K CTAs
 *     that share the group's terms of all column blocks evenly (in column
 *     block order, each CTA takes the tail of one block's terms, whole
 *     blocks and the head of the next; every run starts its multiplier
 *     recurrence afresh); 0 = one CTA per column block, operator and
 *     col_parts run; -1 = the default: K = the device's SMs on square
 *     grids of 128 and 512 points, twice that at 768, else 0.
 * vofl_get_schedule reports the schedule in use, defaults resolved (also
 * while a batch steps the context).
 * Only fused 2D contexts have one (VOFL_EUNSUPPORTED elsewhere).  A context
 * can join a batch whose members of its size are on the same schedule
 * (vofl_batch_tune_transform). */
typedef struct {
  int wide_cols;
  int wide_rows;
  int col_parts;
  int group;
  int fuse_forward;
  int wide_fwd;
  int row_split;
  int col_pack;
} vofl_schedule;
VOFL_API int vofl_set_schedule(vofl_ctx* ctx, const vofl_schedule* sched);
VOFL_API int vofl_get_schedule(vofl_ctx* ctx, vofl_schedule* sched);

/* Library version string. */
VOFL_API const char* vofl_version(void);

/* Self-test of the failure path of device waits (no counterpart in the
 * paper).  Every wait inside the kernels (on TMA copy completion, and the
 * grid-wide barrier of the cooperative forward launch) is bounded by a
 * clock budget: when it runs out the kernel sets an error word, drains
 * what it issued and returns, and vofl_sync() reports VOFL_ETIMEDOUT.  This
 * launches one kernel that waits on an mbarrier nothing completes and one
 * of two CTAs whose second CTA never reaches the grid barrier, each with a
 * ~1 ms budget; *gave_up is set to 1 when both waits gave up as designed.
 * It faults and hangs nothing; the device stays usable.  Synchronous. */
VOFL_API int vofl_selftest_bounded_wait(int* gave_up);

/* Test hook for the out-of-memory paths (no counterpart in the paper).
 * With k > 0, the k-th device allocation the library makes from now on
 * (counting every context, batch and solver allocation of the process)
 * fails as if the device were out of memory, once; k = 0 cancels a pending
 * failure.  Each entry point that allocates then frees what it allocated
 * in that call and returns VOFL_ENOMEM, leaving the context (or batch) as
 * it was.  Process-wide; not for use while other threads allocate.
 * Returns the number of allocations that were still pending before the
 * call (0 when none). */
VOFL_API int64_t vofl_debug_fail_alloc(int64_t k);

/* Memory-checker stand-in (no counterpart in the paper).  When the
 * environment holds VOFL_DEBUG_CANARY=1 at the library's first device
 * allocation, every device buffer the library allocates gets 64 KB pads of
 * a known byte on both sides; a kernel writing up to 64 KB past either end
 * of a buffer changes a pad.  Pads are checked when a buffer is freed and
 * by this call, which synchronises the device and returns the number of
 * buffers found with changed pads (live ones checked now, freed ones when
 * they were freed), or -1 when the mode is off.  *live_buffers (may be
 * NULL): the live padded buffers.  poke = 1 first overwrites one byte of
 * the newest live buffer's end pad from the host (the test that the check
 * sees a change).  Debug use only: every allocation and free synchronises
 * the device. */
VOFL_API int64_t vofl_debug_canaries(int64_t* live_buffers, int poke);

/* ------------------------------------------------------------------------
 * Batches: many independent 2D simulations advanced together.
 *
 * Each simulation is an ordinary context (VOFL_F32, VOFL_IMPL_FUSED, square
 * 2D grid of 64, 128, 256, 512, 768 or 1024 points per side) with its model
 * and state (and optionally a source) set; a batch borrows it and advances
 * it by the leap-frog step of Eq. (1.1) (Eq. (3.4), with the Taylor start
 * for a context that has not stepped yet) with the operators of Eq. (2.13),
 * exactly as vofl_step on the context alone would, bit for bit.  Contexts
 * of a batch may differ in grid size, model, M, dt, source and in how far
 * they have run.  The batch queues its work on its own stream (the one
 * given, or one it creates); every kernel of a step runs once per grid size
 * (or per chunk of simulations of that size, see vofl_batch_tune), so small
 * grids that cannot fill the GPU alone fill it together.  The paper
 * steps one simulation at a time; batching is a throughput layer on top.
 * ------------------------------------------------------------------------ */
typedef struct vofl_batch vofl_batch;

/* New empty batch on the current GPU.  cuda_stream: a cudaStream_t or NULL
 * (the batch creates its own non-blocking stream).  Returns VOFL_OK,
 * VOFL_EINVAL (out is NULL) or VOFL_ECUDA. */
VOFL_API int vofl_batch_create(vofl_batch** out, void* cuda_stream);

/* Wait for the batch's queued work, hand every context back (they stay
 * valid, at the state reached) and free the batch. */
VOFL_API void vofl_batch_destroy(vofl_batch* b);

/* Message of the last error on the batch. */
VOFL_API const char* vofl_batch_last_error(const vofl_batch* b);

/* Add a context; it steps with time step dt (> 0; a context that has
 * already stepped must keep its dt).  Until it is removed, every other
 * entry point on the context returns VOFL_ESTATE (vofl_destroy removes it
 * first).  *slot (may be NULL) receives an id for vofl_batch_remove.
 * Returns VOFL_OK, VOFL_EINVAL, VOFL_ESTATE (model or state not set, or
 * already in a batch), VOFL_EUNSUPPORTED (not a fused FP32 square 2D
 * context of a batched size, or a context of the general model) or
 * VOFL_ECUDA. */
VOFL_API int vofl_batch_add(vofl_batch* b, vofl_ctx* ctx, double dt, int* slot);

/* Remove the context of `slot`; its own stream waits for the batch's
 * queued work, so vofl_get_state on it then sees every step taken.
 * Returns VOFL_OK or VOFL_EINVAL (unknown slot). */
VOFL_API int vofl_batch_remove(vofl_batch* b, int slot);

/* Number of contexts in the batch. */
VOFL_API int vofl_batch_size(const vofl_batch* b);

/* Advance every context of the batch by nsteps >= 0 steps (asynchronous,
 * replayed from CUDA graphs captured on first use and after each change of
 * membership or schedule).  Returns VOFL_OK, VOFL_EINVAL or VOFL_ECUDA. */
VOFL_API int vofl_batch_step(vofl_batch* b, int64_t nsteps);

/* Non-blocking: 1 if the batch's queued steps have finished, 0 if not,
 * < 0 on a CUDA error. */
VOFL_API int vofl_batch_query(vofl_batch* b);

/* Kernels one batch step launches under the current membership and
 * schedule (>= 0), or a negative status. */
VOFL_API int64_t vofl_batch_kernels_per_step(vofl_batch* b);

/* Wait for the batch's stream; VOFL_ETIMEDOUT if a bounded device wait of
 * any member gave up (as vofl_sync), VOFL_ECUDA on a CUDA error. */
VOFL_API int vofl_batch_sync(vofl_batch* b);

/* Autotune the schedule on the live batch: per grid size, the number of
 * simulations per launch (1, 2, 4, 8, 16 or all), then whether sizes run on
 * parallel graph branches, each candidate timed over `reps` two-step graph
 * replays (CUDA events) by coordinate search.  The members' states (both
 * wavefield buffers, L2 u^{n-1} and the step counter) are saved first and
 * put back afterwards, so tuning leaves every simulation where it was.
 * Allocates a temporary copy of those states.  *ms_per_step (may be NULL)
 * receives the best time of one batch step.  Blocks until done. */
VOFL_API int vofl_batch_tune(vofl_batch* b, int reps, double* ms_per_step);

/* Time one batch step of the current schedule (CUDA events over `reps`
 * two-step graph replays after one warm-up), from a saved copy of the
 * members' states that is put back afterwards (as vofl_batch_tune).
 * Blocks until done. */
VOFL_API int vofl_batch_time(vofl_batch* b, int reps, double* ms_per_step);

/* The schedule in use: *parallel = 1 if sizes run on parallel branches;
 * up to cap (size, simulations per launch) pairs (0 = all of that size).
 * Returns the number of pairs. */
VOFL_API int vofl_batch_get_schedule(const vofl_batch* b, int* parallel, int* sizes, int* chunks, int cap);

/* Set the schedule directly (as vofl_batch_get_schedule reports it). */
VOFL_API int vofl_batch_set_schedule(vofl_batch* b, int parallel, const int* sizes, const int* chunks, int n);

/* Transform schedules of a batch (vofl_set_schedule; no counterpart in the
 * paper).  The batched launches of one grid size follow one transform
 * schedule: that of the size's first member; a later member of the size
 * whose context is on another schedule is refused (VOFL_EUNSUPPORTED), so
 * every member gives the bits of its context stepped alone.
 * vofl_batch_tune_transform searches, size by size, the line transforms of
 * each pass, the column runs, the terms per group (at most the members'
 * own) and the runs per row, then the launch layout (as vofl_batch_tune),
 * timing `reps` batch steps per candidate from a saved copy of the state
 * that is put back; it then gives every member its size's schedule (results
 * change in the last bits, within the FP32 tolerance; a member stepped alone
 * afterwards keeps the batch's arithmetic).  *ms_per_step: the best time.
 * vofl_batch_get_transform reports the schedule of grid edge n (VOFL_EINVAL
 * when the batch has no member of that size). */
VOFL_API int vofl_batch_tune_transform(vofl_batch* b, int reps, double* ms_per_step);
VOFL_API int vofl_batch_get_transform(const vofl_batch* b, int n, vofl_schedule* out);

/* Allocation-free variant of vofl_apply_pair for small 2D grids.  The paper
 * has no counterpart: it is a deployment aid for callers that may not
 * allocate device memory when they need the operator (an outside allocator
 * owns the GPU memory budget, cudaMalloc/cudaFree would synchronise the
 * device inside a latency-critical loop, or the caller is a callback that
 * must not enter the CUDA allocator).
 *
 * Computes out1 = (-Delta)^{1+gamma} u and out2 = (-Delta)^{1/2+gamma} u on
 * the periodic box [0,lx) x [0,ly) with nx x ny points (x fastest), with
 * Taylor power M (0..40), exactly as a context created with VOFL_F32 /
 * VOFL_IMPL_FUSED and vofl_set_gamma would.  gamma_dev: nx*ny doubles in
 * [0, 1/2); u_dev, out1_dev, out2_dev: nx*ny floats; all device pointers on
 * the current device; out1_dev or out2_dev may be NULL (not both).
 * stream: a cudaStream_t or NULL.
 *
 * No device memory is allocated: every intermediate lives in one file-scope
 * device array of 6 MiB that each GPU loading the library keeps until the
 * process exits.  Limits: nx, ny in {64, 128, 256} with (nx, ny) one of the
 * fused shapes (64x64, 128x128, 256x256, 256x128, 128x256); larger or
 * other shapes return VOFL_EUNSUPPORTED before any device work.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  The call is
 * synchronous: it waits on `stream` twice, once to read the grid mean of
 * gamma back and once at the end, after the outputs are written, to read
 * the kernels' error word; when it returns VOFL_OK the outputs are
 * complete.  All calls share the one array, so calls that overlap on the
 * GPU (other streams, other host threads) race and must be serialised by
 * the caller; the array keeps the last call's contents.  Each call clears
 * the two words that must start at zero (the step counter and the error
 * word) on `stream` before its kernels run; everything else in the array
 * is written before it is read.
 * Returns VOFL_OK, VOFL_EINVAL (bad arguments or gamma outside [0,1/2)),
 * VOFL_EUNSUPPORTED (shape beyond the limit), VOFL_ETIMEDOUT (a bounded
 * device wait inside the kernels gave up; the outputs are then incomplete)
 * or VOFL_ECUDA. */
VOFL_API int vofl_apply_pair_2d_noalloc(int nx, int ny, double lx, double ly, int M,
                                        const double* gamma_dev, const float* u_dev,
                                        float* out1_dev, float* out2_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VOFL_H */
