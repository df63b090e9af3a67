/*
 * vegas.h -- C ABI of the GB300-native VEGAS library (libgvegas.so).
 *
 * The library runs the data-parallel hot path of the method of
 * J. M. Campbell, R. K. Ellis, W. T. Giele, "A Multi-Threaded Version of
 * MCFM" (arXiv:1503.06182): VEGAS iterations whose events are evaluated
 * independently and then all combined before the grid is optimised
 * (Abstract; Section 2.1), with results independent of how the events are
 * spread over threads (Section 2.2).  Here the events of one iteration are
 * spread over the SMs of one GPU; sums are exact integer fixed-point sums,
 * so results are bit-identical for any launch shape.
 *
 * Conventions
 *  - Every function returns an int status: VEGAS_OK (0) or a negative
 *    VEGAS_E* code; vegas_strerror() describes it.  On error, output
 *    arguments are left unspecified unless stated otherwise.
 *  - All pointer arguments are HOST pointers unless marked "device".  Output
 *    buffers are owned and sized by the caller.  The library owns the device
 *    memory behind a context, except where the caller hands it a workspace.
 *  - Grids are row-major, one row per axis: edges[a*(nbins+1) + i],
 *    0 = e_0 < e_1 < ... < e_nbins = 1.
 *  - Work is enqueued on the context's CUDA stream (its own, or the one set
 *    with vegas_set_stream); blocking calls synchronise that stream only.
 *  - A context is not thread-safe; distinct contexts may be used from
 *    distinct host threads.
 */
#ifndef GVEGAS_VEGAS_H
#define GVEGAS_VEGAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define VEGAS_OK 0
#define VEGAS_EINVAL (-1)     /* invalid argument (dimension, size, id, parameter) */
#define VEGAS_ENOMEM (-2)     /* device or pinned-host allocation failed */
#define VEGAS_ECUDA (-3)      /* a CUDA runtime call failed */
#define VEGAS_EGRID (-4)      /* grid edges not 0 = e_0 < ... < e_N = 1 */
#define VEGAS_ENONFINITE (-5) /* non-finite weights were seen (results computed with them set to 0) */
#define VEGAS_EDEVICE (-6)    /* a device-side check failed */
#define VEGAS_ESTATE (-7)     /* checkpoint buffer does not match this context */

/* ---- integrands (synthetic stand-ins for the paper's H+2 jets, Section 3.2) ---- */
#define VEGAS_GAUSS 0 /* params[1] or [2]: sigma [, shift].  g = prod_a exp(-(x_a-1/2)^2/(2 sigma^2))
                         - shift (shift 0 if not given; weights can then be negative); ndim >= 1 */
#define VEGAS_DY 1    /* params[10]: sqrt_s, M_Z, Gamma_Z, sin2_thetaW, alpha, m_lo, m_hi, a, b, N.
                         LO pp -> gamma*,Z -> mu+ mu- in pb with toy densities
                         f_q = N x^a (1-x)^b, f_qbar = 0.2 N x^a (1-x)^(b+4); ndim >= 4 */
#define VEGAS_EE3J 2  /* params[1 or 2]: y_cut [, sqrt_s = 91.1876].
                         e+e- -> q qbar g, (x1^2+x2^2)/((1-x1)(1-x2)) with y_ij > y_cut; ndim >= 5 */
#define VEGAS_DY_NLO 3 /* params[11]: the ten of VEGAS_DY, then beta.  An NLO-shaped stand-in
                          for the paper's 13-dimensional NLO integral (Section 3.2): the
                          Drell-Yan weight of x_0..x_3 times exp(beta cos(2 pi x_k)) / I0(beta)
                          for every further axis k (each factor integrates to 1, so the
                          integral is the Drell-Yan cross section); ndim >= 4; not batched */

/* ---- limits ---- */
#define VEGAS_MAX_DIM 16
#define VEGAS_MIN_BINS 2
#define VEGAS_MAX_BINS 1024
#define VEGAS_MAX_DIM_BINS 4096 /* ndim * nbins */
#define VEGAS_NGRAD 5           /* Drell-Yan gradient: M_Z, Gamma_Z, sin2_thetaW, a, b */
#define VEGAS_TILE 1024         /* canonical events per tile */

/* ---- options (vegas_set_option / vegas_batch_set_option) ---- */
#define VEGAS_OPT_ALPHA 0     /* grid damping exponent alpha >= 0 (default 1.5) */
#define VEGAS_OPT_PRECISION 1 /* 0 = FP64 integrand (default), 1 = FP32 integrand; the sums are
                                 exact integer sums in both forms */
#define VEGAS_OPT_ADAPT 2     /* 1 = refine the grid after every iteration (default), 0 = frozen */
#define VEGAS_OPT_EPT 3       /* events per thread of the fill kernel: 0 = autotuned (trial
                                 launches per shape; 4 unless another candidate is more than 2%
                                 faster), or 1, 2, 4, 8 (8 only for ndim <= 8: VEGAS_EINVAL
                                 above).  Results do not depend on it. */
#define VEGAS_OPT_NONFINITE 4 /* 0 = return VEGAS_ENONFINITE if any weight is not finite (default),
                                 1 = set such weights to 0 and count them silently */
#define VEGAS_OPT_GRAPH 5     /* 1 = replay the iterations as one CUDA graph (default), 0 = plain launches */
#define VEGAS_OPT_TIMING 6    /* 1 = time every fill and reduce kernel with CUDA events */
#define VEGAS_OPT_BATCH_ID 7  /* Philox batch word of this context (default 0; < 2^24) */
#define VEGAS_OPT_PDL 8       /* 1 = chain the kernels of consecutive iterations with programmatic
                                 dependent launches (default), 0 = ordinary stream order */
#define VEGAS_OPT_STRAT 9     /* 1 = VEGAS+ adaptive stratified sampling (see vegas_strat_get),
                                 0 = plain VEGAS (default) */
#define VEGAS_OPT_BETA 10     /* VEGAS+ damping of the allocation: 0, 0.25, 0.5, 0.75 (default), 1 */
#define VEGAS_OPT_BATCH_GRID 11 /* batches only: each work list's persistent grid in eighths of
                                   its resident CTAs, 1..8; 0 = tuned (default) */

/* ---- kernel ids for vegas_kernel_time ---- */
#define VEGAS_KERNEL_FILL 0   /* per-event kernel */
#define VEGAS_KERNEL_REDUCE 1 /* combination of all events, iteration record, grid optimisation */
#define VEGAS_KERNEL_REFINE 2 /* grid optimisation alone: runs inside the reduce kernel, so it
                                 reports 0 launches */

typedef struct vegas_ctx vegas_ctx;
typedef struct vegas_batch vegas_batch;

/* Create a context for ndim axes with nbins bins each and a uniform grid
 * (e_i = i/nbins).  seed keys the Philox4x32-10 generator: event e of global
 * iteration t uses counter (e, t, batch<<8 | block) and key (seed) -- the
 * "groups of pseudo-random numbers" handed to each event (Section 2.2).
 * Allocates the device memory of the context on the current device.
 * EINVAL unless 1 <= ndim <= 16, 2 <= nbins <= 1024, ndim*nbins <= 4096. */
int vegas_init(int ndim, int nbins, uint64_t seed, vegas_ctx** out);

/* Release the context and its device memory (NULL is ignored). */
void vegas_free(vegas_ctx* ctx);

/* Set one VEGAS_OPT_* option.  EINVAL for an unknown key or value. */
int vegas_set_option(vegas_ctx* ctx, int key, double value);

/* Use the given CUDA stream (cudaStream_t, not owned; NULL = the legacy
 * default stream) for all further work of the context. */
int vegas_set_stream(vegas_ctx* ctx, void* stream);

/* Device workspace for the per-tile partials and per-iteration records of a
 * call with (ncall, itmx): bytes needed. */
int vegas_workspace_size(const vegas_ctx* ctx, int64_t ncall, int itmx, size_t* bytes);

/* Hand the context a caller-owned DEVICE buffer of `bytes` bytes (256-byte
 * aligned) to use as workspace instead of allocating its own; NULL reverts to
 * library allocation.  The buffer must outlive its use by the context. */
int vegas_set_workspace(vegas_ctx* ctx, void* device_ptr, size_t bytes);

/* One "stage": itmx VEGAS iterations of ncall events each (Section 2.1;
 * Section 3.2 runs a 4 x 1,000 warm-up stage and a 10 x 10,000 production
 * stage).  Per iteration k: I_k = sum w / C, sigma_k^2 = (sum w^2/C - I_k^2)/(C-1);
 * the grid is refined after every iteration unless VEGAS_OPT_ADAPT = 0.  The
 * grid and the global iteration counter persist across calls; the
 * combination restarts with every call:
 *   integral = sum(I_k/sigma_k^2)/sum(1/sigma_k^2), error = sum(1/sigma_k^2)^(-1/2),
 *   chi2_dof = sum((I_k - integral)^2/sigma_k^2)/(itmx - 1)  (0 when itmx = 1);
 * iterations with sigma_k = 0, if any, are averaged alone with error 0.
 * integrand_id / params: VEGAS_GAUSS, VEGAS_DY, VEGAS_EE3J, VEGAS_DY_NLO as above.
 * per_iter (nullable): itmx x (I_k, sigma_k).  Blocking.
 * Errors: EINVAL (ncall < 2, itmx < 1, unknown id, wrong nparams or a
 * parameter outside its range), ENOMEM, ECUDA, ENONFINITE (results valid,
 * non-finite weights counted as 0). */
int vegas_iterate(vegas_ctx* ctx, int64_t ncall, int itmx, int integrand_id, const double* params,
                  int nparams, double* integral, double* error, double* chi2_dof,
                  double* per_iter);

/* Enqueue the same stage without waiting; results stay on the device until
 * vegas_fetch.  params are copied before the call returns. */
int vegas_launch(vegas_ctx* ctx, int64_t ncall, int itmx, int integrand_id, const double* params,
                 int nparams);

/* Wait for the last vegas_launch and copy its results (any pointer may be
 * NULL).  per_iter: itmx x (I_k, sigma_k).  nonfinite (nullable): number of
 * non-finite weights seen. */
int vegas_fetch(vegas_ctx* ctx, double* integral, double* error, double* chi2_dof,
                double* per_iter, int64_t* nonfinite);

/* Copy the current grid (ndim x (nbins+1)) to host memory. */
int vegas_grid_get(const vegas_ctx* ctx, double* edges);

/* Replace the grid.  EGRID unless every axis has e_0 = 0, e_nbins = 1 and
 * strictly increasing edges; the grid is unchanged on error. */
int vegas_grid_set(vegas_ctx* ctx, const double* edges);

/* Checkpoint: the grid, the global iteration counter, the seed and the
 * options, in an opaque host buffer of vegas_state_size() bytes.  Restoring
 * it into a context of the same ndim/nbins reproduces the continuation
 * bit-exactly.  ESTATE if the buffer does not belong to such a context. */
int vegas_state_size(const vegas_ctx* ctx, size_t* bytes);
int vegas_state_get(const vegas_ctx* ctx, void* buf, size_t bytes);
int vegas_state_set(vegas_ctx* ctx, const void* buf, size_t bytes);

/* Drell-Yan gradient d sigma / d(M_Z, Gamma_Z, sin2_thetaW, a, b) by a
 * hand-written adjoint (reverse sweep) of the event weight: itmx iterations
 * of ncall events on the current grid, held fixed, with the same event
 * streams a forward stage started at the same iteration counter would use
 * (weights are recomputed, not stored).  Per iteration G_kp = mean dw/dtheta_p;
 * combined with the forward weights 1/sigma_k^2 (their own dependence on
 * theta is not differentiated).  grad, grad_err: VEGAS_NGRAD values.
 * integral/error (nullable): the forward estimate on the same events.
 * per_iter_grad (nullable): itmx x VEGAS_NGRAD x (G_kp, sigma_Gkp).
 * The iteration counter advances by itmx.  EINVAL unless integrand_id is
 * VEGAS_DY. */
int vegas_adjoint(vegas_ctx* ctx, int64_t ncall, int itmx, int integrand_id, const double* params,
                  int nparams, double* grad, double* grad_err, double* integral, double* error,
                  double* per_iter_grad);

/* Diagnostics on single events at the current grid: for each of the n event
 * indices, the weight w = J g(x) and its bins (n x ndim int32), using
 * iteration counter value `iteration`.  Does not advance anything. */
int vegas_eval_events(vegas_ctx* ctx, int integrand_id, const double* params, int nparams,
                      uint32_t iteration, const int64_t* events, int64_t n, double* w,
                      int32_t* bins);

/* Raw Philox4x32-10 words of events first_event .. first_event+n-1 at
 * iteration `iteration` and batch word `batch`: out is n x ndim uint32. */
int vegas_rng_words(uint64_t seed, uint32_t iteration, uint32_t batch, int64_t first_event,
                    int64_t n, int ndim, uint32_t* out);

/* No-allocation variant of vegas_rng_words (the paper has no counterpart).
 * For callers that cannot allocate device memory: a process whose device
 * memory a caching allocator holds (cudaMalloc from another library then
 * fails although the cache has room), or latency-critical code that cannot
 * take the device-wide synchronisation of cudaFree.  Same arguments, same
 * words, but written through a fixed buffer of VEGAS_NOALLOC_MAX_WORDS uint32
 * words (1 MiB) in the library's device image, held by every GPU that loads
 * the library until the process exits; out is host memory owned by the
 * caller.  n * ndim > VEGAS_NOALLOC_MAX_WORDS: VEGAS_EINVAL, nothing launched.
 * The first call on a device, with that device current, does the set-up: it
 * looks up the buffer's device address and loads the kernel (a call with
 * n = 0 does only that); make it before any stream capture begins.  The
 * address is kept for the life of the process: calls must not cross a
 * cudaDeviceReset (or any release of the device's primary context).  The
 * buffer is shared by every call on a device and keeps the last call's
 * words: calls that overlap on one device race on it, so the caller must
 * serialise them.  Nothing in the buffer has to start at zero.  Blocking;
 * runs on the legacy default stream.  VEGAS_ECUDA: a CUDA call failed. */
#define VEGAS_NOALLOC_MAX_WORDS (1 << 18)
int vegas_rng_words_noalloc(uint64_t seed, uint32_t iteration, uint32_t batch,
                            int64_t first_event, int64_t n, int ndim, uint32_t* out);

/* Measurement helper (no counterpart in the paper): the rate of one
 * arithmetic pipe of the current GPU at its present clock, the denominator of
 * the per-event kernels' rooflines (they are bound by plain arithmetic, not by
 * a dense contraction or by HBM).  A probe kernel runs 8 independent chains of
 * one instruction per thread, 8 resident 256-thread CTAs per SM, for about
 * `ms` milliseconds (0 < ms <= 10000; the round count is calibrated first):
 *   VEGAS_PIPE_FFMA  FP32 fused multiply-add, 2 flops each;
 *   VEGAS_PIPE_DFMA  FP64 fused multiply-add, 2 flops each;
 *   VEGAS_PIPE_IMAD  32-bit integer multiply-add, 1 op each;
 *   VEGAS_PIPE_MUFU  FP32 base-2 exponential approximation, 1 op each.
 * *ops_per_s receives flops (or ops) per second.  Uses the legacy default
 * stream and allocates a small output buffer.  VEGAS_EINVAL for an unknown
 * pipe or duration, VEGAS_ECUDA if a CUDA call failed. */
#define VEGAS_PIPE_FFMA 0
#define VEGAS_PIPE_DFMA 1
#define VEGAS_PIPE_IMAD 2
#define VEGAS_PIPE_MUFU 3
int vegas_pipe_peak(int pipe, double ms, double* ops_per_s);

/* FP64 sums of the last iteration: (sum w, sum w^2, d[ndim*nbins]), with
 * d[a*nbins + i] = sum of w^2 over the events in bin i of axis a. */
int vegas_last_sums(const vegas_ctx* ctx, double* sums);

/* Histogram of an observable, filled while integrating (the differential
 * distributions of Section 3.2, there the di-jet mass; here one observable
 * per integrand):
 *   VEGAS_GAUSS: x_0;  VEGAS_DY and VEGAS_DY_NLO: the dilepton mass
 *   m_ll = sqrt(tau s) in GeV;  VEGAS_EE3J: the thrust max(x1, x2, x3).
 * vegas_hist_set(ctx, nbins, lo, hi): nbins equal bins over [lo, hi)
 * (1 <= nbins <= VEGAS_HIST_MAX_BINS, finite lo < hi), plus an underflow bin
 * (below lo, or not a number) and an overflow bin (hi and above): the bin of
 * a value v >= lo is 1 + trunc((v - lo) * (nbins / (hi - lo))), computed in
 * the integrand's precision (FP32 in the FP32 form).  nbins = 0 switches the
 * histogram off.  Every later vegas_iterate / vegas_launch stage fills it:
 * per iteration k and bin b, H_kb = sum_{events in b} w / C and
 * V_kb = (sum_{b} w^2 / C - H_kb^2)/(C-1), from sums that are exact integer
 * sums rounded once to FP64 (so bit-identical for every launch shape); the
 * stage's iterations are combined with the weights of the integral,
 * u_k = 1/sigma_k^2 (or, if any sigma_k is 0, 1 for those iterations and 0
 * for the others):
 *   value_b = sum_k u_k H_kb / sum_k u_k,
 *   error_b = sqrt(sum_k u_k^2 V_kb) / sum_k u_k,
 * so the nbins + 2 values add up to the stage's integral.  With a histogram
 * the fill runs at 4 events per thread (VEGAS_OPT_EPT is not used).  The
 * histogram is not part of a checkpoint, and vegas_adjoint does not fill it.
 * vegas_hist_get(ctx, value, error, last_sums): after such a stage (blocks
 * until it is done), copies value and error (nbins + 2 each, underflow first,
 * overflow last) and last_sums (2 x (nbins + 2): the last iteration's sum w
 * per bin, then its sum w^2); any pointer may be NULL.  EINVAL if no
 * histogram is set, or the last stage did not fill it. */
#define VEGAS_HIST_MAX_BINS 1000
int vegas_hist_set(vegas_ctx* ctx, int nbins, double lo, double hi);
int vegas_hist_get(vegas_ctx* ctx, double* value, double* error, double* last_sums);

/* VEGAS+ (VEGAS_OPT_STRAT = 1): adaptive stratified sampling on the VEGAS map
 * (Lepage, J. Comput. Phys. 439 (2021) 110386; a later form of the VEGAS
 * method of Section 2.1).  For a stage of ncall events (8 <= ncall <= 2^30):
 *   - the map's input cube is cut into nh = s^ndim hypercubes, s the largest
 *     integer with 4 s^ndim <= ncall and s^ndim <= 2^22; hypercube h has the
 *     base-s digits c_a of h as coordinates;
 *   - hypercube h gets n_h >= 2 events, numbered hypercube by hypercube
 *     (uniform floor(ncall/nh) at the start); event e's word on axis a is
 *     floor((c_a 2^32 + r_a)/s), r_a its Philox word; F = J g as in VEGAS;
 *   - per hypercube, the sample variance v_h of F; the iteration's estimate
 *     I_k = sum_e F C/(nh n_h) / C and sigma_k^2 = sum_h v_h/n_h / nh^2; the
 *     grid is trained on F^2/(nh n_h) per event;
 *   - the next allocation: n_h = max(2, floor(ncall d_h / sum d)),
 *     d_h = v_h^(beta/2) (formed in FP32 from correctly rounded operations),
 *     so an iteration has between 2 nh and ncall + 2 nh events.
 * The allocation persists across stages with the same ncall (and is frozen
 * with VEGAS_OPT_ADAPT = 0); VEGAS+ excludes histograms and vegas_adjoint
 * (EINVAL).  The fill runs at 4 events per thread.
 * vegas_strat_get: after a VEGAS+ stage (blocks until done), s, nh, the
 * allocation for the next iteration (counts, nh int32, nullable) and the last
 * iteration's v_h (var, nh doubles, nullable).  EINVAL before any.
 * vegas_strat_set: the allocation for stages of ncall events (counts: nh
 * values >= 2 summing to at most ncall + 2 nh; EINVAL otherwise).
 * The allocation is not part of a checkpoint: after vegas_state_set the next
 * VEGAS+ stage starts from the uniform allocation, unless one saved with
 * vegas_strat_get is restored with vegas_strat_set. */
int vegas_strat_get(vegas_ctx* ctx, int* nstrat, int64_t* ncubes, int32_t* counts, double* var);
int vegas_strat_set(vegas_ctx* ctx, int64_t ncall, const int32_t* counts);

/* Accumulated device time of the VEGAS_KERNEL_* kernels since the last
 * reset (VEGAS_OPT_TIMING = 1 only); reset != 0 clears that kernel's totals
 * after reading. */
int vegas_kernel_time(vegas_ctx* ctx, int kernel, double* total_ms, int64_t* launches, int reset);

/* The events per thread the last stage used (autotuned or forced). */
int vegas_get_ept(const vegas_ctx* ctx, int* ept);

/* ---- batched integrations (many independent VEGAS runs per launch) ----
 * n integrations of uneven dimension, call count and integrand run as one
 * persistent fill launch per iteration, dimension class (at most 4, 8, 16
 * axes) and integrand over a work list of (integration, tile) items taken
 * largest-first from a device counter, then one reduce and
 * one refine launch serving every integration; the itmx iterations are
 * captured in one CUDA graph (Section 2.1: many independent runs, here
 * sharing one device).  All integrations share nbins and seed.
 * Integration b uses Philox batch word b, so its events are those of a
 * single context with VEGAS_OPT_BATCH_ID = b, and its results are
 * bit-identical to that context's.
 * ndim[n], ncall[n], integrand_id[n], nparams[n]; params: n x VEGAS_MAX_PARAMS
 * doubles (row b holds integration b's parameters).  precision: as
 * VEGAS_OPT_PRECISION. */
#define VEGAS_MAX_PARAMS 16
int vegas_batch_create(int n, const int* ndim, const int64_t* ncall, const int* integrand_id,
                       const double* params, const int* nparams, int nbins, uint64_t seed,
                       int precision, vegas_batch** out);
void vegas_batch_free(vegas_batch* b);
/* Keys: VEGAS_OPT_ALPHA, VEGAS_OPT_ADAPT, VEGAS_OPT_NONFINITE, VEGAS_OPT_GRAPH
 * as for a context; VEGAS_OPT_EPT 0 (autotune), 4 or 8.  The first stage
 * tunes the launch shape by timing one iteration's fills, side by side as in
 * a stage: events per thread (4 or 8, unless VEGAS_OPT_EPT fixes them) and
 * each work list's persistent grid (all, 3/4 or 1/2 of its resident CTAs,
 * unless VEGAS_OPT_BATCH_GRID fixes it); results do not depend on the choice.  The precision is fixed at creation
 * (VEGAS_EINVAL otherwise). */
int vegas_batch_set_option(vegas_batch* b, int key, double value);
int vegas_batch_set_stream(vegas_batch* b, void* stream);
/* itmx iterations of every integration; integral/error/chi2_dof: n values;
 * per_iter (nullable): n x itmx x (I_k, sigma_k).  Blocking. */
int vegas_batch_iterate(vegas_batch* b, int itmx, double* integral, double* error,
                        double* chi2_dof, double* per_iter);
/* Edges of integration `index`: ndim[index] x (nbins+1) doubles. */
int vegas_batch_grid_get(const vegas_batch* b, int index, double* edges);

/* Human-readable text of a status code (static storage). */
const char* vegas_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* GVEGAS_VEGAS_H */
