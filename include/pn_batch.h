/*
 * pn_batch.h -- C ABI of the B300 batched post-Newtonian inspiral integrator.
 *
 * Problem (arXiv:0908.3889, Herrmann et al. 2009, Sec. II):  for every binary
 * black hole i, integrate the PN equations of motion Eqs. (1)-(4) -- the
 * orbital frequency omega (Eq. 1), the spins S1, S2 precessing as
 * dS_i/dt = Omega_i x S_i (Eqs. 2, 4) and the orbital axis L-hat (Eq. 3) --
 * with total mass M = m1 + m2 = 1, S_i = chi_i m_i^2 S_i-hat, from a circular
 * orbit at omega_0 with L-hat = z-hat (Sec. V) up to omega_f, with the
 * Dormand-Prince 5(4) method at error tolerance 5e-7 and first step h = 10
 * (Sec. II).  No binary depends on another (Sec. I), so one call
 * integrates a whole batch on one GPU.
 *
 * Conventions for every entry point:
 *  - Return value: PN_OK (0) or a negative PN_E_* code.  Per-binary failures
 *    are not call errors: they are reported in outputs.status[i].  After an
 *    error pn_last_error() describes it.
 *  - Device pointers are caller-owned CUDA device memory (e.g. torch tensors),
 *    float64 unless stated, one value per binary ("structure of arrays"),
 *    each array at least n elements long and 8-byte aligned.  The library
 *    never frees or retains them beyond the call's stream work.
 *  - Calls are ordered on the stream given to pn_batch_init and return
 *    without waiting for the GPU, except where a call says it synchronises.
 *  - A pn_batch is not thread-safe: one host thread at a time per handle.
 */
#ifndef PN_BATCH_H
#define PN_BATCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PN_ABI_VERSION 3

/* ---- return codes ---- */
#define PN_OK 0
#define PN_E_ARG (-1)           /* invalid argument (NULL, n out of range, bad parameter) */
#define PN_E_CUDA (-2)          /* a CUDA runtime call or kernel launch failed */
#define PN_E_NOMEM (-3)         /* device or host allocation failed */
#define PN_E_UNIMPLEMENTED (-4) /* option the library does not support */
#define PN_E_CHECK (-5)         /* debug build only: a device bounds check failed (pn_last_error names the site) */

/* ---- per-binary status (outputs.status) ---- */
#define PN_ST_OK 0
#define PN_ST_MAX_STEPS 1   /* attempt budget params.max_steps exhausted */
#define PN_ST_H_UNDERFLOW 2 /* step size fell below params.h_min after a rejection */
#define PN_ST_NONFINITE 3   /* the state or the error estimate became NaN / Inf */
#define PN_ST_BAD_INPUT 4   /* non-finite input, m_i <= 0, |m1+m2-1| > 1e-12, chi outside [0,1],
                               omega_0 <= 0, omega_f <= omega_0, or | |L-hat_0| - 1 | > 1e-12 */
#define PN_ST_LAND_MAXIT 5  /* the stop at omega_f did not converge in land_max_iter retakes */
#define PN_ST_RUNNING 6     /* pn_batch_integrate_budget / pn_batch_resume: the call's attempt budget ran
                               out; the binary's full state is kept for pn_batch_resume, and the outputs
                               hold its current state */

/* ---- parameter enums ---- */
#define PN_FP64 0  /* everything in FP64 */
#define PN_MIXED 1 /* right-hand side and its stage inputs in FP32; the state increment and the error
                      estimate as compensated FP32 sums, the error norm in FP32; state and step
                      control in FP64 */
#define PN_MIXED_DS 2 /* right-hand side, its stage inputs and the error estimate in double-single
                         (pairs of FP32, ~48-bit significand) on the FP32 pipe; state accumulation,
                         error norm and step control in FP64 */

#define PN_STOP_LAND 0        /* stop exactly on omega_f (default) */
#define PN_STOP_FIRST_CROSS 1 /* stop at the first accepted state with omega >= omega_f */

#define PN_THETA_BCV2 0       /* 3PN: theta-hat multiplies eta once (default reading) */
#define PN_THETA_AS_PRINTED 1 /* 3PN: theta-hat eta^2, as the paper's Eq. (1) prints it */

#define PN_ORDER_INPUT 0  /* lanes take the binaries in input order */
#define PN_ORDER_LENGTH 1 /* lanes take them sorted by predicted length, longest first (default);
                             no result depends on the order */

#define PN_SCHED_AUTO 0       /* use the autotuned choice if any, else persistent */
#define PN_SCHED_PLAIN 1      /* one grid pass: BPT binaries per thread, fixed assignment */
#define PN_SCHED_PERSISTENT 2 /* persistent grid, lanes refill from a device work queue */

/* PN terms of Eq. (1) and the precession of Eqs. (2)-(4) (term_mask bits) */
#define PN_TERM_1PN (1u << 0)  /* -(743 + 924 eta)/336 x^{2/3} */
#define PN_TERM_SO (1u << 1)   /* 1.5PN spin-orbit sum */
#define PN_TERM_TAIL (1u << 2) /* +4 pi x */
#define PN_TERM_2PN (1u << 3)  /* non-spin 2PN */
#define PN_TERM_SS (1u << 4)   /* 2PN spin-spin */
#define PN_TERM_25PN (1u << 5)
#define PN_TERM_3PN (1u << 6)  /* 3PN including the log */
#define PN_TERM_35PN (1u << 7)
#define PN_TERM_PREC (1u << 8) /* spin and L-hat precession; off freezes S_i and L-hat */
#define PN_TERM_ALL 0x1ffu

typedef struct {
  /* Integrator (Sec. II gives the 5e-7 tolerance and h0 = 10; the rest are readings):
   * a step is accepted when the RMS over the 10 state components of
   * e_i / (atol + rtol * max(|y_i|, |y_new_i|)) is <= 1, e = h sum_j (b_j - bhat_j) k_j;
   * the next step is h * clamp(safety * err^(-1/5), fac_min, fac_max), with no growth
   * right after a rejection. */
  double rtol;     /* default 5e-7 */
  double atol;     /* default 5e-7 */
  double h0;       /* first step, default 10 (units of M) */
  double safety;   /* default 0.9 */
  double fac_min;  /* default 0.2 */
  double fac_max;  /* default 10 */
  double h_min;    /* default 1e-10: a rejected step below this gives PN_ST_H_UNDERFLOW */
  double land_tol; /* stop: Newton retakes until |omega - omega_f| <= land_tol * omega_f, then a
                      first-order move along f lands omega on omega_f; default 1e-7 */
  int64_t max_steps;     /* cap on attempts (accepted + rejected + landing retakes); default 1e6 */
  int32_t land_max_iter; /* retakes allowed at the stop, default 8 */
  int32_t stop_mode;     /* PN_STOP_* */
  uint32_t term_mask;    /* PN_TERM_* bits, default PN_TERM_ALL */
  int32_t theta_mode;    /* PN_THETA_* */
  int32_t fixed_step;    /* 1: accept every attempt with h = h0 (convergence studies), default 0 */
  int32_t precision;     /* PN_FP64, PN_MIXED or PN_MIXED_DS */
  int32_t schedule;      /* PN_SCHED_* */
  int32_t block;         /* threads per block (multiple of 32, <= 256); 0 = autotuned / default */
  int32_t bpt;           /* plain schedule: binaries each thread integrates in turn, 1 or 2;
                            0 = autotuned / default 1 */
  int32_t ckpt_every;    /* adjoint: accepted steps between state checkpoints, default 64 */
  int32_t order;         /* PN_ORDER_*: the order in which lanes take the binaries, default
                            PN_ORDER_LENGTH.  The lanes of a warp run in lock-step, so binaries of
                            similar length in one warp waste fewer lane-steps; the outputs are the
                            same bits in either order.  pn_integrate_noalloc ignores it. */
} pn_params;

/* Inputs, one value per binary (device pointers).  Read-only for
 * pn_batch_integrate / _adjoint / _stats; written by pn_batch_sample.
 * s1*, s2*: spin directions S_i-hat (their raw components are used:
 * S_i(0) = chi_i m_i^2 S_i-hat); l*: L-hat at omega_0 (unit); masses with
 * m1 + m2 = 1. */
typedef struct {
  double *m1, *m2, *chi1, *chi2;
  double *s1x, *s1y, *s1z, *s2x, *s2y, *s2z;
  double *lx, *ly, *lz;
  double *omega0, *omega_f;
} pn_inputs;

/* Outputs, one value per binary (device pointers, written by the call).
 * S1, S2, L: final state (L is the evolved L-hat, not renormalised);
 * omega, t: final frequency and time (t from 0 at omega_0);
 * n_acc / n_rej / n_land: accepted steps (the final landing step counts once),
 * rejected attempts, landing retakes (int32);  status: PN_ST_* (int32);
 * dot_s1s2 = S1.S2/(|S1||S2|), dot_ls1 = L.S1/(|L||S1|), dot_ls2 likewise
 * (Sec. V's scalar products; NaN when a spin is zero).  On PN_ST_BAD_INPUT
 * the state, t and dots are NaN and the counters 0. */
typedef struct {
  double *S1x, *S1y, *S1z, *S2x, *S2y, *S2z, *Lx, *Ly, *Lz;
  double *omega, *t;
  int32_t *n_acc, *n_rej, *n_land, *status;
  double *dot_s1s2, *dot_ls1, *dot_ls2;
} pn_outputs;

/* Distribution for pn_batch_sample (Sec. V: isotropic spin directions by
 * Marsaglia's method; masses, spin magnitudes and omega_0 as configured). */
typedef struct {
  int32_t q_mode;   /* q = m1/m2: 0 fixed q_lo, 1 uniform [q_lo,q_hi], 2 log-uniform [q_lo,q_hi] */
  int32_t chi_mode; /* chi_i: 0 fixed chi_lo, 1 uniform [chi_lo,chi_hi] (independent per BH) */
  double q_lo, q_hi, chi_lo, chi_hi;
  double omega0_lo, omega0_hi; /* omega_0 uniform in [lo, hi] (equal bounds: fixed) */
  double omega_f;
} pn_dist;

/* Cotangents of a scalar loss with respect to the outputs (device pointers,
 * length n; a NULL pointer means zero).  Used by pn_batch_adjoint. */
typedef struct {
  const double *dot_s1s2, *dot_ls1, *dot_ls2;
  const double *Lx, *Ly, *Lz;
  const double *S1x, *S1y, *S1z, *S2x, *S2y, *S2z;
  const double *t;
} pn_cotangents;

/* Gradients written by pn_batch_adjoint (device pointers, length n): the loss
 * differentiated with respect to the raw components of S1-hat(0), S2-hat(0)
 * and the mass ratio q = m1/m2 (with M = 1 and chi_i fixed).  Two optional
 * groups (NULL first pointer: group not written; all-or-none within a group):
 *  - *_tan: the spin gradients projected onto the tangent plane of the sphere
 *    at each initial direction s, g - (g . s) s / |s|^2;
 *  - *_dtheta, *_dphi: derivatives with respect to the polar and azimuthal
 *    angles of each initial direction, s = |s| (sin t cos p, sin t sin p,
 *    cos t) with |s| held fixed (at a pole, p = 0 is taken). */
typedef struct {
  double *s1x, *s1y, *s1z, *s2x, *s2y, *s2z;
  double *q;
  double *s1x_tan, *s1y_tan, *s1z_tan, *s2x_tan, *s2y_tan, *s2z_tan;
  double *s1_dtheta, *s1_dphi, *s2_dtheta, *s2_dphi;
} pn_grads;

/* Batch statistics (host struct filled by pn_batch_stats). */
typedef struct {
  int64_t n;
  int64_t count_by_status[8];
  int64_t acc_total, rej_total, land_total;
  int32_t acc_min, acc_max;
  int32_t attempts_min, attempts_max;
  /* Pearson r (Sec. V A) of initial vs final scalar products over binaries
   * with status OK and finite products: S1-hat.S2-hat, L-hat.S1-hat, L-hat.S2-hat. */
  double pearson_s1s2, pearson_ls1, pearson_ls2;
  int64_t pearson_count;
  double mean_final_s1s2, std_final_s1s2;
  /* Device time of the last pn_batch_integrate / pn_batch_adjoint (ms, CUDA events). */
  double ms_last_integrate, ms_last_adjoint;
} pn_stats;

/* Result of pn_batch_autotune. */
typedef struct {
  int32_t schedule, block, bpt;
  int32_t n_candidates; /* shapes timed by this call (0: the shape came from the process's cache) */
  double best_ms;     /* time of the chosen configuration on the tuning prefix */
  int64_t n_tuned;    /* binaries in the tuning prefix */
} pn_tune_result;

/* Quantities for the analysis entry points (Sec. V's scalar products of unit vectors). */
#define PN_Q_FINAL_S1S2 0 /* S1-hat.S2-hat at omega_f */
#define PN_Q_FINAL_LS1 1  /* L-hat.S1-hat at omega_f */
#define PN_Q_FINAL_LS2 2  /* L-hat.S2-hat at omega_f */
#define PN_Q_INIT_S1S2 3  /* S1-hat.S2-hat at omega_0 (from the inputs) */
#define PN_Q_INIT_LS1 4   /* L-hat.S1-hat at omega_0 */
#define PN_Q_INIT_LS2 5   /* L-hat.S2-hat at omega_0 */

/* Histogram specification: 1-D if ny == 1 (quantity_y ignored), else 2-D with
 * x along the slow index (counts[kx * ny + ky]).  A value in [lo, hi] goes to
 * bin min(nb - 1, floor((x - lo) * (nb / (hi - lo)))); others are not counted.
 * nx * ny <= 8192. */
typedef struct {
  int32_t quantity_x, quantity_y;
  int32_t nx, ny;
  double x_lo, x_hi, y_lo, y_hi;
} pn_hist_spec;

typedef struct pn_batch pn_batch; /* opaque: owns only its workspace */

/* Library ABI version (PN_ABI_VERSION). */
int pn_abi_version(void);

/* Fill *p with the defaults listed in pn_params. */
void pn_params_default(pn_params *p);

/* Create a batch context for up to n_max binaries per call on the current
 * CUDA device and the given stream (cudaStream_t, NULL = legacy default).
 * Allocates the small device workspace (queue head, reduction buffers, the
 * logarithm table), uploads the table and waits for the device, and records
 * *p.  Errors: PN_E_ARG (NULL out/p, n_max < 1,
 * bad parameters), PN_E_CUDA, PN_E_NOMEM.  *out is NULL on failure. */
int pn_batch_init(pn_batch **out, int64_t n_max, const pn_params *p, void *cuda_stream);

/* Replace the parameters (same validation as pn_batch_init). */
int pn_batch_set_params(pn_batch *b, const pn_params *p);

/* Draw n binaries of the distribution d into the caller's input arrays, from
 * counter-based SplitMix64 uniforms keyed by (seed, binary index, draw number)
 * (Sec. V; Marsaglia 1972 for the directions; L-hat = z-hat).  Draw j of
 * binary i is the j-th output of the SplitMix64 stream seeded with the i-th
 * output of the stream seeded with `seed`, as a 53-bit uniform; draws 0..3
 * give q, chi1, chi2, omega_0 and draws 4.. the Marsaglia pairs for S1-hat
 * then S2-hat.  Errors: PN_E_ARG (NULL pointers, n > n_max, bad d), PN_E_CUDA. */
int pn_batch_sample(pn_batch *b, uint64_t seed, const pn_dist *d, int64_t n, const pn_inputs *in);

/* Masses from mass ratios, the first step of the per-binary set-up (Sec. II:
 * M = m1 + m2 = 1): m1[i] = q[i]/(1 + q[i]), m2[i] = 1/(1 + q[i]) for
 * i < n, each correctly rounded from the rounded 1 + q[i] (the rounding
 * pn_batch_sample uses).  q, m1, m2: caller-owned device arrays of n doubles;
 * m1 and m2 may be two rows of a pn_inputs block.  Asynchronous on b's
 * stream.  q <= 0 or non-finite q gives masses that pn_batch_integrate then
 * reports as PN_ST_BAD_INPUT.  Errors: PN_E_ARG (NULL b or, for n > 0, a NULL
 * array; n outside [0, n_max]), PN_E_CUDA. */
int pn_batch_masses(pn_batch *b, int64_t n, const double *q, double *m1, double *m2);

/* Device time of the last pn_batch_integrate / _integrate_budget / _resume /
 * _integrate_host call on b (ms, CUDA events on the batch's stream): *ms_call
 * the whole call (set-up, integration kernel, output epilogue), *ms_kernel the
 * integration kernel alone (either pointer may be NULL).  Waits for that call
 * to finish.  A call with n = 0 launches no kernel: *ms_kernel is then the
 * kernel time of the last call that did, or NaN if none has.  Errors: PN_E_ARG
 * (NULL b, or no integration call yet), PN_E_CUDA. */
int pn_batch_timing(pn_batch *b, double *ms_call, double *ms_kernel);

/* Integrate binaries 0..n-1 of *in and write *out (asynchronous).
 * 0 <= n <= n_max (n = 0 does nothing).  Errors: PN_E_ARG (NULL pointers,
 * n out of range), PN_E_CUDA (launch failure).  Uses the schedule, block and
 * binaries-per-thread of the parameters, or the autotuned choice for 0. */
int pn_batch_integrate(pn_batch *b, int64_t n, const pn_inputs *in, pn_outputs *out);

/* Bounded integration with resume.  pn_batch_integrate_budget starts binaries
 * 0..n-1 like pn_batch_integrate, but each binary makes at most `budget`
 * Dormand-Prince attempts (budget >= 1) in this call; a binary still running
 * then gets status PN_ST_RUNNING, its current state in *out, and its complete
 * integrator state (y, f(y), t, step size, landing bracket, counters, flags)
 * kept in library-owned device memory (n_max x 24 doubles + 6 int32,
 * allocated on first use).  pn_batch_resume continues exactly those binaries
 * of 0..n-1 whose status in *out is PN_ST_RUNNING, for at most `budget` more
 * attempts each (budget = 0: until they finish); other binaries are not
 * touched.  The same *in, *out and parameters must be passed to the calls of
 * one run, and no other integration of the batch may come between them (the
 * set-up table is shared).  A run continued until no binary is PN_ST_RUNNING
 * gives results bit-identical to one pn_batch_integrate call.  Bounded calls
 * keep each kernel launch short (for time slicing, or for inspecting or
 * copying the state between calls).  Asynchronous; count the binaries still
 * running with pn_batch_stats (count_by_status[PN_ST_RUNNING]).
 * Errors: PN_E_ARG (NULL pointers, n out of range, budget < 1 for the first
 * call or < 0 for resume, a resume whose params.precision differs from the
 * bounded run's), PN_E_NOMEM, PN_E_CUDA. */
int pn_batch_integrate_budget(pn_batch *b, int64_t n, const pn_inputs *in, pn_outputs *out, int32_t budget);
int pn_batch_resume(pn_batch *b, int64_t n, const pn_inputs *in, pn_outputs *out, int32_t budget);

/* Same as pn_batch_integrate with HOST input and output arrays: copies the
 * inputs to the library's device staging buffers (allocated on first use,
 * n_max binaries), integrates, copies the outputs back and synchronises the
 * stream (it is pn_batch_integrate_host_async followed by pn_batch_host_wait).
 * Page-locked host memory gives the fastest copies.  Errors: PN_E_ARG,
 * PN_E_NOMEM, PN_E_CUDA. */
int pn_batch_integrate_host(pn_batch *b, int64_t n, const pn_inputs *host_in, pn_outputs *host_out);

/* The same as pn_batch_integrate_host without the final wait: enqueues the
 * input copy (on a library copy-in stream), the integration (on the batch's
 * stream) and the output copy (on a library copy-out stream) and returns.
 * The call alternates between two device staging sets (each allocated on
 * first use, n_max binaries), so consecutive calls overlap: a call's input
 * copy runs during the previous call's integration and its output copy during
 * the next call's.  Until pn_batch_host_wait returns, the caller must not
 * change *host_in's arrays nor read *host_out's, for every call made since the
 * last wait.  Results are those of pn_batch_integrate_host.  Errors: PN_E_ARG,
 * PN_E_NOMEM, PN_E_CUDA. */
int pn_batch_integrate_host_async(pn_batch *b, int64_t n, const pn_inputs *host_in, pn_outputs *host_out);

/* Wait until every pn_batch_integrate_host_async call made on b has copied its
 * outputs to the host (and the batch's stream is idle).  Errors: PN_E_ARG,
 * PN_E_CUDA. */
int pn_batch_host_wait(pn_batch *b);

/* The right-hand side f(y) of Eqs. (1)-(4) (arXiv:0908.3889 Sec. II) at n
 * given states, evaluated by the integration kernels' own device function in
 * the batch's precision (PN_FP64, PN_MIXED: FP32, PN_MIXED_DS: double-single)
 * and term mask / theta mode, with the coefficients formed from (m1[i], m2[i])
 * (M = 1, so m1 + m2 = 1 is expected; nothing is validated).  y and f are
 * DEVICE arrays of 10 x n doubles, component-major: component c of state i at
 * [c * n + i], in the order omega, S1 (3), S2 (3), L-hat (3); m1, m2 hold n
 * doubles.  The caller owns every array.  States with |omega| outside
 * [2^-126, 2^128) (the FP32 normal range, in every precision) give
 * non-finite rates.  Asynchronous on the batch's stream.  Errors: PN_E_ARG
 * (NULL batch or pointer, n < 0), PN_E_CUDA. */
int pn_batch_eval_rhs(pn_batch *b, int64_t n, const double *m1, const double *m2, const double *y, double *f);

/* Time the candidate launch shapes of the current precision -- plain schedule x
 * {64, 128, 256} threads x {1, 2} binaries per thread, persistent schedule x
 * {64, 128, 256} threads -- on the first min(n, 262144) binaries of *in (writing
 * *scratch_out), keep the fastest for later calls with schedule/block/bpt = 0,
 * and report it in *res (may be NULL).  The process keeps each result in a cache
 * keyed by the device, the precision, the tuning prefix's size, the parameters
 * that change the work (tolerances, step control, stop, PN terms, lanes' order)
 * and a 64-bit fingerprint of the prefix's inputs; a call that finds its key
 * there times nothing, takes the cached shape and reports n_candidates = 0 with
 * the cached best_ms (the scratch outputs are then not written).  Synchronises.
 * Errors: PN_E_ARG, PN_E_CUDA. */
int pn_batch_autotune(pn_batch *b, int64_t n, const pn_inputs *in, pn_outputs *scratch_out,
                      pn_tune_result *res);

/* Reverse-mode gradient of L = sum_i gbar_i . outputs_i with respect to
 * S1-hat(0), S2-hat(0) and q, through the accepted Dormand-Prince steps of
 * the forward integration with the step sizes held fixed and the stop at
 * omega_f differentiated as an implicit function (the landing step size h*
 * solves omega(h*) = omega_f).  Runs the forward pass, records the accepted
 * step sizes and a checkpoint every params.ckpt_every accepted steps in
 * library-owned device memory (grown on demand), then sweeps backwards one
 * checkpoint segment at a time, recomputing the segment's states.  Each lane
 * of the sweep (at most a few tens of thousands on one GPU) keeps the
 * recomputed segment: ckpt_every x 306 doubles in the FP64 sweep (the stage
 * states with the right-hand side's intermediate values, ~6 GB for a full
 * B300 grid at the default stride), ckpt_every x 60 in the double-single one.  Requires
 * PN_STOP_LAND and adaptive steps.  With precision PN_FP64 the forward pass
 * and the backward sweep are FP64; with PN_MIXED_DS both run in double-single
 * arithmetic on the FP32 pipe, the forward pass being pn_batch_integrate's
 * PN_MIXED_DS attempt (faster; gradients within ~1e-8 relative of the FP64
 * ones, the same steps taken); PN_MIXED is refused.  The forward pass takes
 * the binaries in params.order, as pn_batch_integrate does.  Binaries whose
 * status is not PN_ST_OK get NaN gradients.  If out is not NULL the forward
 * outputs are written there too (in PN_MIXED_DS, the double-single run's).  Errors: PN_E_ARG, PN_E_NOMEM, PN_E_CUDA,
 * PN_E_UNIMPLEMENTED (other modes). */
int pn_batch_adjoint(pn_batch *b, int64_t n, const pn_inputs *in, const pn_cotangents *gbar,
                     pn_grads *grad, pn_outputs *out);

/* Reduce outputs 0..n-1 (and the initial scalar products of *in) into *host
 * (counts per status, step totals, Pearson r of Sec. V A).  Synchronises.
 * Errors: PN_E_ARG, PN_E_CUDA. */
int pn_batch_stats(pn_batch *b, int64_t n, const pn_inputs *in, const pn_outputs *out, pn_stats *host);

/* pn_batch_stats for several ensembles integrated together in one call (the
 * parameter sweeps of Sec. V B-D: one ensemble per mass ratio, spin magnitude
 * or omega_0, concatenated along the binary index): segment k is binaries
 * host_offsets[k] .. host_offsets[k + 1] - 1 and its statistics go to
 * host[k].  host_offsets: n_seg + 1 non-decreasing host int64 values in
 * [0, n_max] (an empty segment gives n = 0 and NaN Pearson r); host: n_seg
 * caller-owned records.  One reduction launch covers every segment.
 * n_seg = 0 does nothing.  Synchronises.  Errors: PN_E_ARG (NULL pointers,
 * n_seg outside [0, 65535], bad offsets), PN_E_NOMEM (the scratch for the
 * partial records, grown on demand and kept by the batch), PN_E_CUDA. */
int pn_batch_stats_segments(pn_batch *b, int32_t n_seg, const int64_t *host_offsets, const pn_inputs *in,
                            const pn_outputs *out, pn_stats *host);

/* Histogram of outputs 0..n-1 (Sec. V A: 20 and 100 bins of the final
 * S1-hat.S2-hat; 79 x 79 bins of initial vs final; Sec. V B's KS test uses
 * fine 1-D bins).  nx * ny <= 4,194,304 bins.  Only binaries with status OK
 * and finite values count.  Writes nx * ny counts to host_counts and
 * synchronises.  Errors: PN_E_ARG (bad spec, NULL pointers), PN_E_CUDA. */
int pn_batch_histogram(pn_batch *b, int64_t n, const pn_inputs *in, const pn_outputs *out, const pn_hist_spec *spec,
                       int64_t *host_counts);

/* One-sample Kolmogorov-Smirnov test of binned values against the uniform
 * distribution on [lo, hi] (Sec. V B tests the final S1-hat.S2-hat this way):
 * counts[0..n_bins-1] of equal-width bins, e.g. from pn_batch_histogram (any
 * number of calls summed).  The binned empirical CDF brackets the statistic:
 * d_lo <= D <= d_hi (d_lo is D at the bin edges; with N values in n_bins bins
 * the two differ by at most the largest bin's share).  p_at_d_lo and
 * p_at_d_hi are the asymptotic Kolmogorov p-values at those D (with Stephens'
 * sqrt(N) + 0.12 + 0.11/sqrt(N) scaling).  Host only: needs no GPU or batch.
 * Errors: PN_E_ARG (NULL pointers, n_bins < 1, lo >= hi, a negative count). */
typedef struct {
  int64_t n;              /* number of values (sum of counts) */
  double d_lo, d_hi;      /* bounds on the KS statistic D */
  double p_at_d_lo, p_at_d_hi;
} pn_ks_result;
int pn_ks_uniform(const int64_t *counts, int32_t n_bins, double lo, double hi, pn_ks_result *res);

/* Gaussian kernel density estimate of one quantity (Sec. V A):
 * p(x) = 1/(N h) sum_j K((x - x_j)/h), K(u) = exp(-u^2/2)/sqrt(2 pi), with
 * h = 1.06 sigma N^(-1/5) (sigma the sample standard deviation, N the number of
 * binaries with status OK and a finite value), evaluated at the m points of
 * host_grid (m <= 65536) into host_density; the bandwidth goes to *host_h (may be
 * NULL).  Synchronises.  Errors: PN_E_ARG, PN_E_NOMEM, PN_E_CUDA. */
int pn_batch_kde(pn_batch *b, int64_t n, const pn_inputs *in, const pn_outputs *out, int32_t quantity,
                 const double *host_grid, int64_t m, double *host_density, double *host_h);

/* Release the workspace (waits for the stream).  NULL is ignored. */
void pn_batch_destroy(pn_batch *b);

/* Integrate binaries 0..n-1 like pn_batch_integrate (persistent schedule, 128
 * threads per block) without allocating any device memory, for callers that
 * must not allocate: hosts that give all device memory to their own pool or
 * budget and cannot have a library call cudaMalloc behind their back.  The
 * paper has no counterpart; it is a deployment variant of the same kernels.
 * Scratch (work-queue counter, logarithm table, per-binary set-up table) lives
 * in one fixed area of about 6 MiB inside the library's device image, held
 * on every GPU that loads the library until exit, so n <= 16384 per call
 * (larger n: PN_E_ARG).  No pn_batch is needed: *p, *in and *out are as for
 * pn_batch_init / pn_batch_integrate, and the work is queued on cuda_stream
 * (cudaStream_t, NULL = legacy default) without waiting.  All calls share the
 * area (each call resets what it reads), so calls whose GPU work overlaps race.
 * The first call on a device looks up the area's address, uploads the
 * logarithm table and waits for the device; make that first call before any
 * stream capture.  Errors: PN_E_ARG, PN_E_CUDA; message via pn_last_error(NULL). */
int pn_integrate_noalloc(int64_t n, const pn_params *p, const pn_inputs *in, pn_outputs *out, void *cuda_stream);

/* Self-test of the debug build's device bounds checks; the paper has no
 * counterpart.  The debug build (libpn_b300_debug.so, compiled with -DPN_DEBUG)
 * stands in for a memory checker: its kernels check the indices that come from
 * data (the lanes' permutation of the binaries, scatter positions, histogram
 * bins) and the per-thread shared-memory workspaces against the launch, skip
 * an access that fails its check and record the site, and each entry point
 * that launches device work then waits for it and returns PN_E_CHECK if a
 * check failed (debug builds therefore synchronise and cannot be captured in a
 * CUDA graph).  This call launches one kernel whose single check fails on
 * purpose (it guards no memory access) and returns PN_OK when that failure is
 * reported and cleared, PN_E_CHECK otherwise, PN_E_CUDA on a CUDA error, and
 * PN_E_UNIMPLEMENTED in the release build.  Message via pn_last_error(NULL). */
int pn_debug_selftest(void);

/* Message of the last error on b (or, when b is NULL, of the last failed
 * pn_batch_init or pn_integrate_noalloc on this thread); empty string if none.
 * Valid until the next call. */
const char *pn_last_error(const pn_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* PN_BATCH_H */
