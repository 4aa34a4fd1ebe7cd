/*
 * anova_gb300.h -- C ABI of the GB300 (sm_103a) ANOVA-Gaussian fast summation
 * and kernel ridge regression library (libanova_gb300.so).
 *
 * Method: Nestler, Stoll, Wagner, "Learning in High-Dimensional Feature Spaces
 * Using ANOVA-Based Fast Matrix-Vector Multiplication", arXiv 2111.10140.
 *
 *   K alpha = sum_l eta_l K_l alpha,  (K_l)_{ij} = exp(-||x_i^{W_l} - x_j^{W_l}||^2 / ell^2)
 *     (Sec. 3, Eq. extended_Gaussian_ANOVA_kernel; Sec. 5 weights eta_l)
 *   K_l alpha ~= Phi D Phi^* alpha  (Sec. 4.3), computed per window by the NFFT
 *     fast summation of Sec. 4.2, Eq. (fastsum): Kaiser-Bessel spreading onto a
 *     sigma*n oversampled grid (adjoint NFFT, Eq. adjnfft), FFT, multiplication
 *     by the Fourier coefficients of the periodised kernel, inverse FFT, and
 *     gathering (NFFT, Eq. nfft).
 *   (K + lambda I) alpha = y solved by conjugate gradients (Sec. 2).
 *   s(z) = sum_j alpha_j kappa(z, x_j) at test points (Sec. 4.2 Eq. kernelsum,
 *     Sec. 4.3 "Phi_z D Phi^* alpha").
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" must be CUDA device (or managed) memory on the
 *     current device; "host" pointers are ordinary host memory.  The caller
 *     owns every buffer it passes; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; entry points that must return a host
 *     value (plan creation, CG iteration counts) synchronise that stream.
 *   - Errors are returned as anova_status; no exception crosses the ABI.
 *     anova_last_error() returns a thread-local detail string for the last
 *     failure on the calling thread.
 *   - A plan serves one call at a time: its grids and work buffers are shared
 *     by every call on it, so calls on one plan from several threads (or on
 *     several streams at once) must be serialised by the caller.  Fitted
 *     models and the server state their own rules below.
 *   - Scratch the calls need comes stream-ordered from the device's default
 *     memory pool.  On its first such allocation on a device the library
 *     raises that pool's release threshold to 1 GiB (unless it is higher
 *     already), so freed scratch stays reserved across synchronisations
 *     instead of being unmapped and mapped again by the next call.
 *   - Arrays of points are row-major: point i, feature f at [i*ld + f].
 *   - Multiple right-hand sides are column-major: column r at [r*ld + i].
 */
#ifndef ANOVA_GB300_H
#define ANOVA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct anova_plan anova_plan;   /* opaque; owned by the library */

typedef enum {
    ANOVA_OK = 0,
    ANOVA_EINVAL = 1,    /* bad argument (sizes, windows, ell, n, m, lambda ...) */
    ANOVA_ENOMEM = 2,    /* device allocation failed */
    ANOVA_ECUDA = 3,     /* a CUDA call failed; see anova_last_error() */
    ANOVA_ENOCONV = 4,   /* CG reached maxit; outputs hold the last iterate */
    ANOVA_ERANGE = 5,    /* input outside the supported range */
    ANOVA_ETIMEOUT = 6,  /* a bounded device-side wait expired */
    ANOVA_EBUSY = 7      /* a request refused: its expected queue wait exceeds the server's bound */
} anova_status;

/* precision bitmask for anova_fastsum_plan: which operators the plan holds */
#define ANOVA_FP64  1    /* FP64 spread / FFT / gather */
#define ANOVA_FP32  2    /* FP32 spread / FFT / gather */
#define ANOVA_MIXED 3    /* both: FP32 bulk work with FP64 refinement in CG */

/*
 * anova_fastsum_plan -- build the fast-summation plan for the node set X
 * (Sec. 4.2 scaling of the nodes into the torus, Sec. 4.2 Fourier coefficients
 * of the periodised kernel, Sec. 5 windows and weights).
 *
 *   points   device, N x d FP64, row-major with leading dimension ld >= d.
 *   windows  host, P x 3 int32, 0-based feature indices, unused slots -1;
 *            each window holds 1 to 3 distinct features (Sec. 3 Eq. index_window).
 *            Windows may overlap.
 *   weights  host, P FP64 kernel weights eta_l; NULL means eta_l = 1/P (Sec. 5).
 *   ell      Gaussian width in the units of `points`, kernel exp(-r^2/ell^2).
 *   n        host, P int32 bandwidths (even, >= 4); NULL means 32 for every window.
 *   m        Kaiser-Bessel cutoff (1..12); 2m+2 <= sigma*n is required.
 *   sigma    oversampling factor; sigma*n must be an even integer (2 is usual).
 *   eps_B    regularisation width of the periodised kernel, 0 < eps_B < 1/2
 *            (nodes are scaled into the ball of radius 1/4 - eps_B/2).
 *   p        smoothness of the transition polynomial (degree 2p-1), 1..16.
 *   precision  ANOVA_FP64, ANOVA_FP32 or ANOVA_MIXED.
 *   out      host, receives the plan.
 *
 * The plan copies what it needs (the window coordinates), so `points` may be
 * freed after return.  It synchronises `stream`.  Errors: EINVAL for invalid
 * arguments, ENOMEM, ECUDA.
 */
anova_status anova_fastsum_plan(const double* points, int64_t N, int32_t d, int64_t ld,
                                const int32_t* windows, int32_t P, const double* weights,
                                double ell, const int32_t* n, int32_t m, double sigma,
                                double eps_B, int32_t p, int32_t precision,
                                void* stream, anova_plan** out);

/*
 * anova_fastsum_plan_bins -- anova_fastsum_plan with the bin side of the dense
 * spread / gather kernels chosen per window dimension: bin_side (host, 3
 * int32) for the 1-D, 2-D and 3-D windows, 0 = the default rule.  A side is
 * taken when it is even, the region side + 2m <= 16, the bins fit the binning
 * (at most 32768) and, in 1-D, side + m - 2 < n_os; otherwise the default rule
 * applies (anova_plan_window_bins reports what was taken).  bin_side NULL is
 * anova_fastsum_plan.  The paper fixes no binning: a tuning parameter of the
 * GPU design.  Errors as anova_fastsum_plan.
 */
anova_status anova_fastsum_plan_bins(const double* points, int64_t N, int32_t d, int64_t ld,
                                     const int32_t* windows, int32_t P, const double* weights, double ell,
                                     const int32_t* n, int32_t m, double sigma, double eps_B, int32_t p,
                                     int32_t precision, const int32_t* bin_side, void* stream, anova_plan** out);

/*
 * anova_autotune_bins -- the bin sides (per window dimension) that make the
 * matrix-vector product fastest on this GPU, by measurement: the default rule
 * first, then every admissible side for the 1-D, 2-D and 3-D windows in turn,
 * each timed over `reps` products (FP32 if the precision holds it) after three
 * warm-up products (a GPU tuning step; the paper has no counterpart).
 * Arguments as anova_fastsum_plan; bin_side (host, 3 int32)
 * receives the choice for anova_fastsum_plan_bins (0 = default rule), ms (host
 * or NULL) its time per product.  Builds and frees one plan per candidate;
 * synchronous.  Errors: those of the plan build, EINVAL.
 */
anova_status anova_autotune_bins(const double* points, int64_t N, int32_t d, int64_t ld, const int32_t* windows,
                                 int32_t P, const double* weights, double ell, const int32_t* n, int32_t m,
                                 double sigma, double eps_B, int32_t p, int32_t precision, int32_t reps,
                                 int32_t* bin_side, double* ms, void* stream);

/*
 * anova_autotune_kernels -- on a built plan holding the FP32 operator, the
 * kernel forms that make its FP32 product fastest on this GPU, by measurement
 * (coordinate descent from the plan's current forms, each candidate timed
 * over `reps` products after two warm-up products), left set on the plan.
 * choice (host, 3 int32) receives:
 *   [0] 3-D spread: 0 FP32 FMA, 1 mma.sync 3xTF32, 2 the same with the next
 *       chunk copied (cp.async) during the current MMAs (the default), 3 as 2
 *       with FP16 operands split in three terms (m16n8k16: twice the nodes
 *       per tensor-core instruction; coefficients scaled by max |alpha|, one
 *       extra reduction per product);
 *   [1] 3-D gather: 0 FP32 FMA, 1 mma.sync 3xTF32, 2 tcgen05 one block per
 *       sub-problem group, 3 persistent warp-specialised tcgen05 (the default;
 *       where the problem is too small to fill the GPU it runs as 2);
 *   [2] 1-D / 2-D schedule, as anova_plan_set_overlap & 3.
 * Every form computes the same product to the FP32 bar (1e-5 relative);
 * only speed and rounding differ.
 * ms (host or NULL) receives the chosen forms' time per product.  The tile
 * shapes inside each form are fixed by its instruction (mma.sync m16n8k8,
 * tcgen05 M = 128); the bin side, which sets each sub-problem's region, is
 * tuned by anova_autotune_bins.  Synchronous; drops the plan's captured
 * graphs; must not overlap with other calls on the plan.  The paper has no
 * counterpart: a tuning step of the GPU design.
 * Errors: EINVAL (NULL plan or choice, reps < 1, no FP32 operator, N = 0),
 * those of anova_matvec, ECUDA; on an error the plan keeps its forms.
 */
anova_status anova_autotune_kernels(anova_plan* plan, int32_t reps, int32_t* choice, double* ms, void* stream);

/* anova_plan_set_kernels / anova_plan_get_kernels -- set or read the plan's
 * kernel forms directly (forms: host, 3 int32, coded as the choice of
 * anova_autotune_kernels).  Setting drops the plan's captured graphs and must
 * not overlap with other calls on the plan.  Errors: EINVAL (NULL argument, a
 * form out of range). */
anova_status anova_plan_set_kernels(anova_plan* plan, const int32_t* forms);
anova_status anova_plan_get_kernels(const anova_plan* plan, int32_t* forms);

/*
 * anova_matvec -- out = K alpha with the fast operator (Sec. 4.3, K alpha ~=
 * sum_l eta_l Phi_l D_l Phi_l^* alpha).
 *
 *   dtype  ANOVA_FP64 (alpha, out are double*) or ANOVA_FP32 (float*); the
 *          plan must hold that precision.
 *   alpha  device, nrhs columns of N entries, column r at alpha + r*ld.
 *   out    device, same layout; overwritten.  Must not alias alpha.
 *   nrhs   >= 1; ld >= N.
 * Asynchronous on `stream`.  With nrhs = 1 the plan records the call's launch
 * sequence as a CUDA graph the second time it sees the same (dtype, alpha,
 * out) and replays it from then on (at most 16 graphs per plan, shared with
 * the CG solver, which replays its operator application the same way).  While
 * a call captures, no other host thread may synchronise the whole device
 * (cudaDeviceSynchronize, torch.cuda.synchronize): CUDA refuses that while any
 * stream captures.  Multi-threaded callers switch capture off with
 * anova_plan_set_graphs.  Calls on one plan must not overlap on the GPU: they
 * share the plan's work buffers.  The call does not wait for its kernels, so a
 * bounded wait that gave up inside one (the result is then invalid) shows only
 * in anova_wait_timeouts; the synchronous calls below compare that counter
 * and return ETIMEOUT.
 * Errors: EINVAL.
 */
anova_status anova_matvec(anova_plan* plan, int32_t dtype, const void* alpha, void* out,
                          int32_t nrhs, int64_t ld, void* stream);

/*
 * krr_cg_solve -- solve (K + lambda I) alpha = y by conjugate gradients
 * (Sec. 2; Hestenes-Stiefel, alpha_0 = 0), stopping when the recursive residual
 * satisfies ||r||_2 <= tol ||y||_2 or after maxit iterations.
 *
 *   y, alpha  device FP64, nrhs columns with leading dimension ld >= N.
 *   iters     host, nrhs int32 (may be NULL): iterations used per column.
 *   relres    host, nrhs FP64 (may be NULL): true relative residual
 *             ||y - (K + lambda I) alpha|| / ||y|| recomputed at the end with
 *             the FP64 operator when the plan holds it, else the FP32 one.
 * Plans with ANOVA_FP64 run CG with the FP64 operator; ANOVA_FP32 with the
 * FP32 operator (FP64 vectors and scalars); ANOVA_MIXED runs FP32 inner CG
 * inside FP64 iterative refinement until the FP64 residual meets tol.
 * maxit: 0 .. ANOVA_MAX_CG_ITERS (the residual history lives on the device).
 * Synchronises `stream`.  Errors: EINVAL (lambda <= 0, tol <= 0, maxit out of
 * range ...), ENOCONV (maxit reached; alpha and relres hold the last iterate), ETIMEOUT
 * (a bounded wait inside a kernel gave up during the call, as counted by
 * anova_wait_timeouts; the result is not to be trusted).
 */
#define ANOVA_MAX_CG_ITERS (1 << 24)
anova_status krr_cg_solve(anova_plan* plan, double lambda, const double* y, double* alpha,
                          int32_t nrhs, int64_t ld, double tol, int32_t maxit,
                          int32_t* iters, double* relres, void* stream);

/*
 * krr_predict -- out_i = sum_l eta_l sum_j alpha_j kappa_l(z_i, x_j) at M test
 * points (Sec. 4.3 "s ~= Phi_z D Phi^* alpha").
 *
 *   alpha  device FP64, N coefficients.
 *   Z      device FP64, M x d row-major, leading dimension ldz >= d.
 *   out    device FP64, M entries.
 * Uses the plan's highest precision (FP64 when held).  When a test point maps
 * outside the plan's ball the library builds a temporary frame over X and Z
 * together (the kernel is shift- and scale-invariant in user units), so the
 * call still returns ANOVA_OK.  Synchronises `stream`; allocates its scratch
 * stream-ordered.  Errors: EINVAL (M < 0 or M >= 2^31, ldz < d, missing
 * pointers), ECUDA (a failed allocation included), ETIMEOUT (a bounded wait
 * inside a kernel gave up during the call; out is not to be trusted).
 */
anova_status krr_predict(anova_plan* plan, const double* alpha, const double* Z, int64_t M,
                         int64_t ldz, double* out, void* stream);

/*
 * krr_predict_noalloc -- the same prediction as krr_predict, but the call
 * itself allocates no device memory: no cudaMalloc, cudaFree or allocating
 * library routine runs inside it.  The paper has no counterpart; this entry
 * point exists for callers that cannot allocate while serving a request: a
 * server that admits requests against a fixed device-memory budget (an
 * allocation inside a request could fail or push the process over its budget
 * under load), or a process whose device allocator belongs to another
 * framework (a cudaMalloc here would bypass that allocator's pool and
 * accounting).
 *
 * Arguments and result are those of krr_predict, with these limits:
 *   - M <= 65536 test points per call; larger M returns ANOVA_EINVAL.
 *   - The per-call scratch (test-point coordinates, their binned copy, sort
 *     histograms, per-window results; about 7 MiB at M = 65536) lives in one
 *     8 MiB file-scope device array that every GPU loading the library holds
 *     until the process exits.  The plan's own buffers are used as in
 *     anova_matvec.
 *   - The first call on a device looks up that array's device address (with
 *     the device current) and caches it; make that first call before any
 *     stream capture.
 *   - All calls share the array: calls that overlap on the GPU (other threads,
 *     other streams) race and corrupt each other's results.  Serialise them.
 *   - A test point outside the plan's ball returns ANOVA_ERANGE (krr_predict
 *     would build a joint frame, which needs allocation).
 * Synchronises `stream`: the call reads each window's largest test-point
 * radius back to the host for the ball check, and returns after the result
 * is written.
 */
anova_status krr_predict_noalloc(anova_plan* plan, const double* alpha, const double* Z, int64_t M,
                                 int64_t ldz, double* out, void* stream);

/*
 * anova_direct_matvec -- the exact kernel sum, no fast summation (Sec. 2
 * Eq. mult_with_K; Sec. 4.2 Eq. kernelsum with Z != X), O(M N P) work:
 *   out_i = sum_l eta_l sum_j alpha_j exp(-||z_i^{W_l} - x_j^{W_l}||^2 / ell^2).
 *
 *   Z      device FP64, M x d row-major (ldz >= d); pass X for K alpha.
 *   X      device FP64, N x d row-major (ldx >= d).
 *   windows, weights, ell as in anova_fastsum_plan (weights may be NULL).
 *   dtype  ANOVA_FP64 (all in double) or ANOVA_FP32 (coordinates, exponentials
 *          and per-tile partial sums in float, tile sums in double; relative
 *          error around 1e-6).
 *   alpha  device FP64, N entries; out device FP64, M entries.
 * Allocates nothing; asynchronous on `stream`.  Errors: EINVAL.
 */
anova_status anova_direct_matvec(const double* Z, int64_t M, int64_t ldz, const double* X, int64_t N,
                                 int64_t ldx, int32_t d, const int32_t* windows, int32_t P,
                                 const double* weights, double ell, int32_t dtype, const double* alpha,
                                 double* out, void* stream);

/* ----------------------------------------------------------------------------
 * Window construction upstream of the fast summation.
 * ------------------------------------------------------------------------- */

/*
 * anova_zscore_fit -- per-column mean and standard deviation (divisor N) of the
 * training matrix X (device, N x d row-major, row stride ld >= d, d <= 2048)
 * into mean, sd (device, d each); a constant column gets sd = 1 (Sec. 6.1:
 * columns standardised with training statistics only).  Asynchronous on
 * `stream`.  Errors: EINVAL, ECUDA.
 */
anova_status anova_zscore_fit(const double* X, int64_t N, int32_t d, int64_t ld, double* mean, double* sd,
                              void* stream);

/* X <- (X - mean) / sd column by column, in place (device; training or test
 * rows; Sec. 6.1: test rows take the training statistics).  mean, sd: device,
 * d entries (from anova_zscore_fit).  Asynchronous on `stream`.  Errors:
 * EINVAL (shapes as anova_zscore_fit, missing pointers), ECUDA. */
anova_status anova_zscore_apply(double* X, int64_t N, int32_t d, int64_t ld, const double* mean, const double* sd,
                                void* stream);

/*
 * anova_mis -- mutual information score (nats) of every column of X (device,
 * N x d, ld) with the class labels (device, N int32 in [0, nclass)), Sec. 5.
 * The paper leaves the estimator open; this is the plug-in estimate
 * sum_{q,y} (n_qy / N) ln(N n_qy / (n_q n_y)) over `bins` quantile bins q of the
 * column: a value's fine bin is floor((v - lo) 4096 / (hi - lo)) on the
 * column's [lo, hi] (last bin closed), fine bin j maps to quantile bin
 * floor(bins (2 C_j + c_j) / (2 N)), C_j the count below j, c_j its own.
 * mis: host, d doubles.  nclass <= 64, bins <= 64, d * bins * nclass <= 51200.
 * Synchronous.  Errors: EINVAL (also for labels out of range), ECUDA.
 */
anova_status anova_mis(const double* X, int64_t N, int32_t d, int64_t ld, const int32_t* labels, int32_t nclass,
                       int32_t bins, double* mis, void* stream);

/* anova_mis_fine_bins -- the fine bin floor((v - lo) 4096 / (hi - lo)) (last
 * bin closed, lo / hi the column's minimum and maximum) of every element of X,
 * the integer intermediate of anova_mis, into bins (device, N x d int32,
 * row-major, row stride d).  Asynchronous on `stream`.  Errors: EINVAL (shapes
 * as anova_zscore_fit, missing pointers), ENOMEM, ECUDA. */
anova_status anova_mis_fine_bins(const double* X, int64_t N, int32_t d, int64_t ld, int32_t* bins, void* stream);

/*
 * anova_windows_from_mis -- Sec. 5's grouping: features ranked by score
 * (descending, equal scores by index), scores below `threshold` dropped, the
 * rest in consecutive groups of three; the last group holds the one to three
 * left.  windows: host, 3 * d int32 (-1 padded rows, the layout
 * anova_fastsum_plan takes); P: number of windows (0 if none survive).
 * Host only.  Errors: EINVAL (d < 1, missing pointers, a non-finite score).
 */
anova_status anova_windows_from_mis(const double* mis, int32_t d, double threshold, int32_t* windows, int32_t* P);

/* ----------------------------------------------------------------------------
 * Fitted models (Sec. 4.3).  For fixed coefficients alpha the factor
 * D_l Phi_{X,l}^* alpha of the test-point summation -- alpha spread onto window
 * l's grid and convolved with the kernel's Fourier multiplier -- does not
 * depend on the test points.  krr_model_create computes it once per window;
 * krr_model_predict then bins the test points and gathers from those grids.
 * Same kernels and precision as krr_predict (FP64 when the plan holds FP64).
 * The paper has no model object: this caches a factor of its prediction.
 * ------------------------------------------------------------------------- */
typedef struct krr_model krr_model;

/* plan: must outlive the model and must not change its points; alpha: device,
 * N entries, copied (the caller may free it afterwards).  Synchronous on
 * `stream`; uses the plan's work buffers, so no other call on the plan may run
 * meanwhile.  Errors: EINVAL, ENOMEM, ECUDA. */
anova_status krr_model_create(anova_plan* plan, const double* alpha, void* stream, krr_model** out);

/*
 * out (device, M) <- the model's prediction at Z (device, M rows of ld ldz >=
 * d).  Returns when out is written.  Calls on one model may run concurrently
 * from several host threads on different streams: they read the model's grids
 * and allocate their own scratch (stream-ordered).  A call whose test points
 * leave the plan's ball in some window runs krr_predict (re-framed) on the
 * plan's grids instead, one such call per model at a time.
 * Errors: EINVAL, ECUDA, ETIMEOUT (as krr_predict).
 */
anova_status krr_model_predict(krr_model* model, const double* Z, int64_t M, int64_t ldz, double* out,
                               void* stream);

/* Free the model's grids and coefficients.  NULL is ignored. */
void krr_model_destroy(krr_model* model);

/* Copy the model's coefficients alpha (N doubles, the model's own copy) to
 * `out` (device, N entries), stream-ordered on `stream`.  Errors: EINVAL (NULL
 * model, or NULL out with N > 0), ECUDA. */
anova_status krr_model_alpha(const krr_model* model, double* out, void* stream);

/* ----------------------------------------------------------------------------
 * Batches: many problems and right-hand sides per launch.  The paper fits one
 * problem at a time; a batch runs the fits of Sec. 2 for several problems
 * (own nodes, windows, width, lambda) and several right-hand sides each in
 * lockstep: one launch per (window dimension, region size) spreads every
 * (problem, window, right-hand side), one launch sequence transforms all 3-D
 * grids and one all 1-D / 2-D grids, and the CG vector updates of all systems
 * are one launch each; the iteration is replayed as a CUDA graph.  FP32
 * operator (the plans' FP32 kernels), FP64 CG vectors and scalars.
 *
 * Flat vector layout: problem p's right-hand side r, entry i (the problem's
 * node order) at off[p] + r * N_p + i, off from anova_batch_layout.
 * ------------------------------------------------------------------------- */
typedef struct anova_batch anova_batch;

/*
 * plans: nprob plans holding FP32 (ANOVA_FP32 or ANOVA_MIXED), N >= 1, one
 * cut-off m, every window on the dense kernels and box FFTs (EINVAL names the
 * first that is not); the plans must outlive the batch.  nrhs >= 1,
 * nprob * nrhs <= 65535, at most 65535 (problem, window, right-hand side)
 * instances.  Device memory per instance: the window's grid (n_os^dA FP32),
 * 3-D FFT work (2 n_os^2 n complex), sorted coefficients and results (2 N_p).
 * Synchronous on `stream`.  Errors: EINVAL, ENOMEM, ECUDA.
 */
anova_status anova_batch_create(anova_plan* const* plans, int32_t nprob, int32_t nrhs, void* stream,
                                anova_batch** out);

/* offsets (host, nprob + 1 entries) of the flat layout; offsets[nprob] is its
 * length.  Errors: EINVAL (NULL batch or offsets). */
anova_status anova_batch_layout(const anova_batch* batch, int64_t* offsets);

/* y = K x for every system (device, flat layout; y must not alias x), each
 * problem's fast operator of Sec. 4.3.  Asynchronous on `stream`; calls on one
 * batch must not overlap.  Errors: EINVAL (NULL or aliasing vectors), ECUDA. */
anova_status anova_batch_matvec(anova_batch* batch, const double* x, double* y, void* stream);

/*
 * Solve (K_p + lambda_p I) alpha = y for every (problem p, right-hand side) by
 * CG (Sec. 2; Hestenes-Stiefel, alpha_0 = 0), each system stopping when its recursive
 * residual reaches tol ||y|| or after maxit iterations.  lambda: host, nprob
 * entries >= 0.  y, alpha: device, flat layout.  iters, relres: host, nprob *
 * nrhs entries (system p * nrhs + r) or NULL; relres is recomputed with the
 * batch's FP32 operator (NaN for a system whose CG broke down: with the FP32
 * operator K + lambda I may lose definiteness when lambda is below its
 * rounding).  Systems that stop iterate no more (their kernels exit at once).
 * Returns ENOCONV if a system stopped short of tol, EINVAL for a NULL batch,
 * lambda, y or alpha, y aliasing alpha, tol <= 0 or maxit < 1, ECUDA if a CUDA
 * call fails, ETIMEOUT if a bounded wait inside a kernel gave up during the
 * call (alpha is then not to be trusted).  Synchronous on `stream`; the iteration is
 * captured as a CUDA graph on the second block of iterations (same caveat as
 * anova_matvec on device-wide synchronisation from other threads).
 */
anova_status krr_batch_cg_solve(anova_batch* batch, const double* lambda, const double* y, double* alpha,
                                double tol, int32_t maxit, int32_t* iters, double* relres, void* stream);

/*
 * As krr_batch_cg_solve, to an FP64 residual (CG on (K + lambda I) alpha = y,
 * Sec. 2): every plan must hold FP64 too (ANOVA_MIXED).  Passes: the batched
 * FP32 CG solves the correction equation (K32 + lambda I) dx = r of every open
 * system to 1e-4 relative (less when less is left; at most maxit / 8
 * iterations per pass), and alpha += t dx with the step t that minimises the
 * FP64 residual ||r - t (K64 + lambda I) dx|| (each problem's FP64 operator,
 * anova_matvec), so no pass raises a system's residual.  A system whose
 * residual norm falls by less than 10 % in a pass (its FP32 operator no longer
 * resolves the correction) continues with plain FP64 CG on its correction
 * equation, if CG can reach tol within the iterations left: about
 * 0.5 sqrt(kappa) ln(2 relres / tol) with kappa = (lambda_max(K) + lambda) /
 * lambda, lambda_max(K) from 20 power iterations of the problem's FP64
 * operator.  relres is the recomputed FP64 residual; iters sums the FP32 and
 * FP64 iterations of a system; maxit bounds that sum.  Returns ENOCONV when a
 * system ends above tol (its last iterate kept).  Synchronous on `stream`;
 * allocates its work vectors stream-ordered.  Errors as krr_batch_cg_solve,
 * and ENOMEM when the work vectors cannot be allocated.
 */
anova_status krr_batch_cg_solve_refined(anova_batch* batch, const double* lambda, const double* y, double* alpha,
                                        double tol, int32_t maxit, int32_t* iters, double* relres, void* stream);

/* Free the batch (not its plans).  NULL is ignored. */
void anova_batch_destroy(anova_batch* batch);

/* ----------------------------------------------------------------------------
 * Request server: kernel ridge regression fits (anova_fastsum_plan with
 * ANOVA_MIXED, krr_cg_solve, krr_model_create) and predictions
 * (krr_model_predict) served by worker threads, each on its own CUDA stream.
 * Requests are admitted in arrival order as soon as a worker is free and
 * their device memory fits the budget (a request that alone exceeds the
 * budget runs when nothing else does).  Fits occupy at most
 * n_workers - max(1, n_workers / 4) workers; the others stay free for
 * predictions.  Work of different requests overlaps on the GPU, predictions
 * on one model included.  Fitted models stay on the device until released.
 * Plans made by the server do not capture CUDA graphs (anova_plan_set_graphs),
 * so other threads of the process may synchronise the device at any time.
 * The paper serves no requests; this is the serving form of its fit (Sec. 2)
 * and predict (Sec. 4.3) operations.
 * ------------------------------------------------------------------------- */
typedef struct anova_server anova_server;

/* n_workers in 1..64; hbm_budget_bytes > 0 (device bytes the admitted
 * requests and resident models may hold by the server's estimate).  Starts the
 * worker threads on the current device.  Errors: EINVAL, ENOMEM. */
anova_status anova_server_create(int32_t n_workers, int64_t hbm_budget_bytes, anova_server** out);

/*
 * Queue a fit.  points (device, N x d row-major, ld = d) and y (device, N) must
 * stay valid until anova_server_wait on the returned ticket has returned.
 * windows / n (host, copied), ell, m, eps_B as in anova_fastsum_plan (sigma 2,
 * p 8); lambda, tol, maxit as in krr_cg_solve.  The ticket also names the model.
 * Returns at once; the fit's own errors arrive through anova_server_wait.
 * Errors: EINVAL (NULL server or ticket, P outside 1..256, N < 0, maxit out of
 * range); EBUSY (refused by the fit-wait bound, anova_server_set_fit_wait_bound).
 */
anova_status anova_server_submit_fit(anova_server* server, const double* points, int64_t N, int32_t d,
                                     const int32_t* windows, int32_t P, double ell, const int32_t* n,
                                     int32_t m, double eps_B, double lambda, const double* y, double tol,
                                     int32_t maxit, int64_t* ticket);

/* Queue a prediction at M test points Z (device, M x d) into out (device, M)
 * with the model of fit ticket `model` (waits for that fit if needed); Z and
 * out must stay valid until anova_server_wait on the returned ticket has
 * returned.  Errors: EINVAL (NULL server or ticket, M < 0, `model` not a fit
 * ticket); a prediction whose fit failed or whose model was released
 * completes with EINVAL through anova_server_wait. */
anova_status anova_server_submit_predict(anova_server* server, int64_t model, const double* Z, int64_t M,
                                         double* out, int64_t* ticket);

/* Block until the request is done; result receives its status (its detail in
 * anova_last_error), latency_ms the time from submission to completion;
 * iterations / relres the CG figures of a fit.  Output pointers may be NULL.
 * A prediction's ticket is forgotten after its wait; a fit's stays (it names
 * the model).  Errors: EINVAL (NULL server, unknown ticket). */
anova_status anova_server_wait(anova_server* server, int64_t ticket, anova_status* result, double* latency_ms,
                               int32_t* iterations, double* relres);

/* Drop a fitted model and return its memory to the budget.  `model` is the
 * ticket of a fit whose anova_server_wait has returned (EINVAL for an unknown
 * ticket, a fit still queued or running, or a model already released);
 * predictions still running on it finish first, the last one frees it. */
anova_status anova_server_release(anova_server* server, int64_t model);

/* Copy the coefficients alpha of a served fit (the ticket of a fit whose
 * anova_server_wait has returned OK or ENOCONV) to `out` (device, N doubles),
 * synchronously on `stream`.  Errors: EINVAL (unknown, failed or released
 * fit; NULL out), ECUDA. */
anova_status anova_server_fit_alpha(anova_server* server, int64_t fit, double* out, void* stream);

/*
 * Bound on a fit's expected queue wait, in milliseconds (0, the default: no
 * bound).  When a fit is submitted, the server estimates how long it would
 * wait for a worker: the fits queued ahead of it, plus itself, divided by the
 * rate at which fits that had to wait for a worker have been starting (their
 * last up to 16 starts), so the rate follows the mix of fits and the load of
 * the predictions beside them.  A fit whose estimate exceeds the bound is
 * refused at once: anova_server_submit_fit returns ANOVA_EBUSY and queues
 * nothing.  Until two such starts are recorded there is no rate, and a fit is
 * refused only if it would have to queue.  Fits run on low-priority streams
 * and predictions on high-priority ones (cudaStreamCreateWithPriority), so a
 * prediction's kernels are scheduled ahead of the fits' waiting blocks.
 * Predictions are never refused.  The paper has no counterpart: this keeps
 * the fits the server accepts at a bounded latency when they are offered
 * faster than the GPU can fit them.  Errors: EINVAL (NULL server, negative or
 * non-finite bound).
 */
anova_status anova_server_set_fit_wait_bound(anova_server* server, double max_wait_ms);

/* Latency percentiles of the completed requests, their number, and the budgeted
 * bytes currently held (resident models and running requests).  Output
 * pointers may be NULL.  Errors: EINVAL (NULL server). */
anova_status anova_server_stats(anova_server* server, double* p50_ms, double* p99_ms, int64_t* completed,
                                int64_t* bytes_in_use);

/* Stop the workers and free every model.  Queued requests that have not started
 * are dropped; call this only after every anova_server_wait has returned. */
void anova_server_destroy(anova_server* server);

/* Free every device buffer of the plan.  NULL is ignored. */
void anova_plan_destroy(anova_plan* plan);

/* Static description of a status code. */
const char* anova_status_string(anova_status status);

/* Number of bounded waits inside the library's kernels that gave up (an
 * mbarrier that never completed) since the library was loaded; 0 in normal
 * operation, -1 if it cannot be read.  Such a kernel skips its remaining work,
 * frees its tensor memory and returns. */
int64_t anova_wait_timeouts(void);

/*
 * anova_debug_wait_probe -- checks the bounded-wait path of the library's
 * kernels without a fault: one warp waits on a shared-memory mbarrier that
 * nothing arrives on, polling at most `polls` times (1 .. 2^22, the limit of
 * the kernels' own waits), and reports that it gave up.  The paper has no
 * counterpart; this exists so that the ETIMEOUT path can be tested.  Touches
 * neither anova_wait_timeouts nor any plan.  Synchronises `stream`.
 * Returns ETIMEOUT when the wait gave up (the expected outcome), OK if the
 * barrier completed, EINVAL for polls out of range (checked before any CUDA
 * call), ECUDA if the probe could not run.
 */
anova_status anova_debug_wait_probe(int32_t polls, void* stream);

/* Thread-local detail of the last error on the calling thread ("" if none). */
const char* anova_last_error(void);

/* ----------------------------------------------------------------------------
 * Introspection used by tests and benchmarks.
 * ------------------------------------------------------------------------- */

/*
 * anova_plan_window -- frame and grid of window l (Sec. 4.2 scaled nodes):
 * torus coordinate = scale * (x - centre).  centre (host, 3 doubles, unused
 * entries 0), scale, ell_l = scale * ell, dims (1..3), n, nos = sigma*n; output
 * pointers may be NULL.  Host only.  Errors: EINVAL (NULL plan, l out of range).
 */
anova_status anova_plan_window(const anova_plan* plan, int32_t l, double* centre, double* scale,
                               double* ell_l, int32_t* dims, int32_t* n, int32_t* nos);

/*
 * anova_debug_spread -- spreading step alone for window l (the window step of
 * the adjoint NFFT, Eq. adjnfft): grid (device, nos^dims entries of dtype,
 * centred index u + nos/2 per axis, last axis fastest) receives
 *   g_u = sum_j alpha_j prod_t psi(nos x_{j,t} - u_t),
 * where psi is the Kaiser-Bessel window normalised to psi(0) = 1, i.e. the
 * window phi(t) = sinh(b sqrt(m^2-t^2)) / (pi sqrt(m^2-t^2)) divided by phi(0).
 * alpha: device, N entries of dtype in the user's node order.  Asynchronous on
 * `stream`.  Errors: EINVAL (bad plan, l, dtype the plan does not hold, NULL
 * pointers).
 */
anova_status anova_debug_spread(anova_plan* plan, int32_t l, int32_t dtype, const void* alpha,
                                void* grid, void* stream);

/* Bin side, region side and whether window l runs on the dense kernels (the
 * binning is a GPU design choice; the paper fixes none).  Output pointers may
 * be NULL.  Host only.  Errors: EINVAL (NULL plan, l out of range). */
anova_status anova_plan_window_bins(const anova_plan* plan, int32_t l, int32_t* bin_side, int32_t* region,
                                    int32_t* dense);

/*
 * anova_plan_bin_rule -- the binning a plan would give one window of `dims`
 * features with bandwidth n, cut-off m and oversampling sigma, without a plan
 * and without touching the GPU.  bin_side (host, 3 entries for 1-D / 2-D /
 * 3-D windows, 0 = the default rule, may be NULL) is the request that
 * anova_fastsum_plan_bins takes.  Outputs (host, may be NULL): side = bin side
 * in grid cells, region = side + 2m (the cells a bin's nodes reach along one
 * axis), dense = 1 when the window runs on the dense region kernels (region at
 * most 16 cells, at most 32768 bins), nbins = bins of the window.
 * The default rule: 3-D windows take bins of 2 cells (4 when 2 gives too many
 * bins) while the region stays within 16 cells; 2-D windows bins of 2 cells;
 * 1-D windows bins of 16 - 2m cells (2 on grids too small for that); other
 * windows the generic kernels.  A requested side is taken when it is even, its
 * region stays within 16 cells, the bins number at most 32768 and
 * side + m - 2 < sigma n.
 * The paper fixes no binning; this is the GPU design's rule.
 * Errors: EINVAL for arguments anova_fastsum_plan would reject, or a grid
 * too fine for the binning.
 */
anova_status anova_plan_bin_rule(int32_t dims, int32_t n, int32_t m, double sigma, const int32_t* bin_side,
                                 int32_t* side, int32_t* region, int32_t* dense, int32_t* nbins);
/*
 * anova_debug_diag -- copy window l's FP64 multiplier D_k (host, n^dims
 * doubles, centred index) = b_k / prod_t psihat(k_t)^2 with the normalised
 * window (Sec. 4.3 D = diag(c_k) with the window deconvolution folded in).
 * Synchronous.  Errors: EINVAL (NULL plan or output, l out of range), ECUDA.
 */
anova_status anova_debug_diag(const anova_plan* plan, int32_t l, double* D_host);

/*
 * Stage timing.  When enabled, the library records CUDA events on the launch
 * stream around each stage of the fast summation; anova_stage_times returns
 * the accumulated milliseconds and kernel launch counts per stage since the
 * last call (which resets them):
 *   0 spreading, 1 forward FFT, multiply by D, inverse FFT, 2 gathering,
 *   3 window sum and CG vector kernels (grid clearing is a memset, not timed),
 *   4 the 3-D spread kernel launches alone (part of 0), 5 the 3-D gather
 *   kernel launches alone (part of 2).
 * `ms` and `launches` are host arrays of `cap` entries (either may be NULL);
 * returns the number of stages written (0 for a NULL plan).  Reading
 * synchronises the recorded events.  While timing is on, captured graphs are
 * not replayed.  The paper has no counterpart: a measurement aid.
 * anova_set_profiling errors: EINVAL (NULL plan).
 */
anova_status anova_set_profiling(anova_plan* plan, int32_t enable);
int32_t anova_stage_times(anova_plan* plan, double* ms, int64_t* launches, int32_t cap);

/* Allocation-failure injection, for testing the error paths without a device
 * fault: the k-th device allocation the library makes from now on (k >= 1,
 * counted over all threads) fails as if the device were out of memory, once;
 * k = 0 switches the injection off.  The failing call returns ENOMEM or ECUDA
 * and frees what it had allocated.  Errors: EINVAL (k < 0).  The paper has no
 * counterpart: a test aid. */
anova_status anova_debug_fail_alloc(int64_t k);

/* Device memory in use, for leak checks: free device bytes (cudaMemGetInfo),
 * and the bytes in use and reserved in the current device's default
 * stream-ordered pool (memory the library frees stream-ordered goes back to
 * the pool, which may keep it reserved).  Output pointers may be NULL.
 * Errors: ECUDA.  The paper has no counterpart: a test aid. */
anova_status anova_debug_memory(int64_t* free_bytes, int64_t* pool_used_bytes, int64_t* pool_reserved_bytes);

/* Names of the FP32 3-D spread and gather kernels the plan launches (static
 * strings such as "k_spread3_tc<R>", R standing for the region size), so that
 * a measurement can name the kernel stages 4 and 5 time.  The paper has no
 * counterpart: a measurement aid.  Errors: EINVAL (a NULL argument). */
anova_status anova_plan_dense3_kernels(const anova_plan* plan, const char** spread, const char** gather);

/* Graph capture and replay of anova_matvec / krr_cg_solve on (enable != 0,
 * the default) or off; switching off drops the captured graphs.  The paper has
 * no counterpart: this is a launch-overhead setting.  Errors: EINVAL (NULL
 * plan). */
anova_status anova_plan_set_graphs(anova_plan* plan, int32_t enable);

/* anova_plan_set_tensor_cores -- run the plan's FP32 3-D spread and gather on
 * tensor cores (enable != 0, the default: the contraction of a bin's nodes
 * into its region, and the region against the nodes' weights, as 3xTF32
 * mma.sync / tcgen05 products with FP32 accuracy) or on FP32 FMA kernels
 * (enable = 0), e.g. to compare the two; enable = 2 also moves the 3-D spread
 * from mma.sync to the persistent tcgen05 kernel, for comparison only: it
 * measured slower (0.70 against 0.39 ms on N = 1e6 with three 3-D windows)
 * and less accurate (4.4e-5 against the FP64 direct sum, above the FP32 bar
 * of 1e-5).  enable = 1 restores the default forms (3xTF32 spread with the
 * copy pipeline, persistent tcgen05 gather; anova_plan_set_kernels codes 2
 * and 3), replacing a form chosen by anova_autotune_kernels.  The 1-D / 2-D
 * kernels and batches are not affected.  Drops the plan's captured graphs.
 * Must not overlap with other calls on the plan.  Errors: EINVAL (NULL plan). */
anova_status anova_plan_set_tensor_cores(anova_plan* plan, int32_t enable);

/* anova_plan_set_overlap -- how the FP32 product schedules the 1-D / 2-D
 * windows' chain (spread, box FFT, gather) against the 3-D windows' chain.
 * The two touch disjoint grids and result slices; the plan runs the first on
 * a second stream, forked from and joined back to the call's stream by
 * events.  mode & 3: 0 one stream (no overlap); 1 forked before the 3-D
 * spread is queued; 2 (the default) forked before, queued after the 3-D
 * spread; 3 forked after the 3-D spread has run.  mode & 4: the second stream at the
 * device's highest stream priority instead of its lowest.  A scheduling
 * choice only: the results are the same.  Drops the plan's captured graphs.
 * Must not overlap with other calls on the plan.  Errors: EINVAL (NULL plan,
 * mode outside 0..3 and 5..7). */
anova_status anova_plan_set_overlap(anova_plan* plan, int32_t mode);

#ifdef __cplusplus
}
#endif

#endif /* ANOVA_GB300_H */
