/*
 * ssa.h -- C ABI of the GB300 fast Basic SSA library (libssa_gb300.so).
 *
 * Implements the hot path of "Computation- and Space-Efficient
 * Implementation of SSA" (Korobeynikov): the trajectory-matrix products X v
 * and X^T u by FFT against a cached spectrum of the series (section 4,
 * Algorithms 2 and 3), the Golub-Kahan-Lanczos truncated SVD with full
 * reorthogonalisation and thick restart that they drive (section 3,
 * Algorithm 1), and grouped rank-1 Hankelization by FFT convolution
 * (section 5, Algorithm 4; sections 2.3-2.4 for grouping and diagonal
 * averaging).  The trajectory matrix is never formed.
 *
 * Conventions
 *   - Series f[0..N-1] is the paper's f_1..f_N; window L with 1 < L < N,
 *     K = N - L + 1; X is the L x K Hankel matrix X[i][j] = f[i+j].
 *   - Matrices are column-major doubles; U is L x k, V is K x k.
 *   - Singular values are returned in descending order.  Each pair
 *     (u_i, v_i) is signed so that the entry of u_i with the largest
 *     magnitude is positive (lowest index among equals).
 *   - Every pointer argument may be host memory or device memory of the
 *     current CUDA device; the library detects which.  Buffers are owned by
 *     the caller; handles (plans, decompositions) are owned by the library
 *     until destroyed.  Inputs are never modified.
 *   - All GPU work is issued on opts->stream (NULL = the legacy default
 *     stream).  A call returns after its results are complete, except that
 *     ssa_matvec / ssa_hankelize with only device pointers return once the
 *     work is enqueued on the stream.
 *   - Calls return SSA_OK (0) or a positive error code; ssa_strerror()
 *     names it and ssa_last_error() gives a detail message for the calling
 *     thread.  Handles stay valid after an error.  Calls on one plan are not
 *     thread-safe; use one plan per thread.
 *
 * Precision (see SSA_PREC_*): GB300's FP64 pipe runs at about 1/68 of the
 * FP32 rate, so "F64" results are computed in double-float arithmetic
 * (an unevaluated sum of two floats, ~48 significant bits) on the FP32
 * pipes; inputs and outputs are IEEE doubles.
 */
#ifndef SSA_GB300_H
#define SSA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SSA_OK 0
#define SSA_EINVAL 1      /* invalid argument (sizes, k, groups, pointers) */
#define SSA_ENOMEM 2      /* device allocation failed */
#define SSA_ENOCONV 3     /* Lanczos did not converge within max_restarts; results and residuals are still returned */
/* 4 is not used: no kernel of this library waits on another CTA or device, so there is no bounded wait to run out */
#define SSA_ECUDA 5       /* CUDA runtime error */
#define SSA_ENUMERIC 6    /* non-finite value met (input or overflow) */

/* precision modes */
#define SSA_PREC_F64 0    /* all steps in double-float (FP64-class accuracy) */
#define SSA_PREC_F32C 1   /* FFT products in FP32 with the spectrum multiply compensated
                             (spectrum kept in double-float); reorthogonalisation, the
                             projected SVD and the convergence test stay double-float */

typedef struct ssa_plan_s* ssa_plan_t;
typedef struct ssa_decomp_s* ssa_decomp_t;

typedef struct ssa_opts {
  int precision;      /* SSA_PREC_F64 or SSA_PREC_F32C */
  double tol;         /* convergence: every wanted Ritz residual <= tol * sigma_1 (0 = the precision's default:
                         1e-12 for SSA_PREC_F64, 1e-7 sqrt(log2 M) for SSA_PREC_F32C) */
  int max_restarts;   /* thick restarts before SSA_ENOCONV (default 200) */
  int krylov_dim;     /* Krylov dimension d (0 = min(max(2k, k+32), min(L, K)); at most 510) */
  int keep;           /* Ritz pairs kept per restart (0 = k + ceil((d-k)/5)) */
  uint64_t seed;      /* splitmix64 seed of the starting vector p_0 and breakdown vectors */
  void* stream;       /* cudaStream_t for all GPU work (NULL = default stream) */
  int refine;         /* SSA_REFINE_ON: return each sigma_i as the Rayleigh quotient u_i^T X v_i of the
                         returned vectors, computed with native-FP64 FFT products (k extra products);
                         SSA_REFINE_OFF (default): return the Ritz values of the projected matrix */
  double reorth_skip; /* SSA_PREC_F64 only: skip level tau of the reorthogonalisation ("orthogonalise only
                         when necessary", section 3.2.2).  0 (default): never skip, every new vector is made
                         orthogonal to the basis to working precision.  tau > 0: after the first projection
                         h = Q^T w the rest of the Gram-Schmidt is skipped when w, less its coupling to the
                         newest column, is orthogonal to the older columns to tau relative (and that coupling
                         is at most 100 times the rest of w).  1e-12 skips about half of the passes on
                         well-separated spectra; the basis is then orthogonal only to ~tau, so sigma are
                         accurate to ~tau sigma_1 absolute and vectors of closely spaced sigma to
                         ~tau sigma_1 / gap. */
  int reorth;         /* SSA_REORTH_FULL (default): Gram-Schmidt against the whole basis every half-step.
                         SSA_REORTH_PRO (SSA_PREC_F64 only): partial reorthogonalisation (section 3.2.2)
                         in the first Lanczos cycle: each half-step subtracts its one known coupling,
                         updates estimates of the new vector's inner products with the older ones from
                         the projected matrix, and runs the Gram-Schmidt passes only when an estimate
                         exceeds sqrt(eps) (eps = 2^-46, the double-float product error) and on the step
                         after.  The basis is then orthogonal to ~sqrt(eps): sigma keep full accuracy,
                         vectors and reconstructions ~sqrt(eps) (or ~1e-9 sigma_1 / gap).  The
                         coefficients it leaves out would spoil a thick restart, so a first cycle that
                         does not converge starts over from the same starting vector with full
                         Gram-Schmidt (counted as one restart): choose krylov_dim large enough for one
                         cycle.  reorth_skip is ignored in this mode.
                         SSA_REORTH_NONE (SSA_PREC_F64 only): no reorthogonalisation (section 3.2.1): one
                         cycle of krylov_dim steps (default four times the usual 2k or k + 32, at most
                         510) with no Gram-Schmidt and no restart; the singular values of the projected
                         matrix are filtered by the Cullum-Willoughby test (a simple value that is also a
                         singular value of the projected matrix without its first row is spurious; copies
                         count once), and the first k that pass are returned with unit Ritz vectors.
                         Accuracy is not FP64-class in general: converged means k values passed with
                         residual estimates <= tol sigma_1, else SSA_ENOCONV. */
  int grid_cap;       /* most CTAs of one launch of the persistent reorthogonalisation passes and the
                         cooperative normalisation (0, default: as many as are resident on the whole
                         device).  A caller running several decompositions at once on separate streams
                         gives each a share of the device so that their latency-bound kernels run side
                         by side; results change only by the rounding order of the block sums. */
} ssa_opts_t;

#define SSA_REORTH_FULL 0
#define SSA_REORTH_PRO 1
#define SSA_REORTH_NONE 2

#define SSA_REFINE_OFF 0
#define SSA_REFINE_ON 1

/* Fill *opts with defaults: SSA_PREC_F64, tol 0 (precision default), 200 restarts, seed 0, NULL stream,
 * SSA_REFINE_OFF. */
void ssa_default_opts(ssa_opts_t* opts);

/*
 * Embedding step (section 2.1) without forming X: validate N > 2 and
 * 1 < L < N, pick the FFT length M (the least power of two >= N; any M >= N
 * is exact once M - N zeros separate the two blocks of c, Algorithm 2 step
 * 1) and allocate the plan's device tables.  opts may be NULL (defaults).
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_embed_plan(int64_t N, int64_t L, const ssa_opts_t* opts, ssa_plan_t* out);

/* FFT geometry of a plan: *M (FFT length), *single_cta (1 when each transform runs in one CTA). */
int ssa_plan_info(ssa_plan_t plan, int64_t* M, int* single_cta);

/*
 * Cache the spectrum c-hat = FFT_M(c) of the circulant column
 * c = (f_{N-L+1}, ..., f_N, 0 x (M-N), f_1, ..., f_{N-L}) (Algorithm 2
 * steps 1-2).  f: N doubles.  When L > K the plan works on X^T, the
 * K-trajectory matrix of the same series, so c uses window min(L, K).
 * Errors: SSA_EINVAL (null), SSA_ENUMERIC (non-finite f), SSA_ECUDA.
 */
int ssa_set_series(ssa_plan_t plan, const double* f);

/* Copy the cached spectrum C-hat_0..C-hat_{M/2} (M/2 + 1 values) to re / im (natural order, unscaled). */
int ssa_get_spectrum(ssa_plan_t plan, double* re, double* im);

/*
 * Trajectory-matrix products for nvec vectors (Algorithm 2 for transpose =
 * 0: y_j = X x_j, x_j of length K, y_j of length L; Algorithm 3 for
 * transpose = 1: y_j = X^T x_j, x_j of length L, y_j of length K).
 * x and y hold the nvec vectors back to back.  Requires ssa_set_series.
 * Errors: SSA_EINVAL, SSA_ECUDA.
 */
int ssa_matvec(ssa_plan_t plan, int transpose, const double* x, double* y, int nvec);

/*
 * Truncated SVD step (section 2.2 via section 3): the k leading singular
 * triples of X by Golub-Kahan-Lanczos bidiagonalisation (Algorithm 1) with
 * reorthogonalisation against the whole basis on both sides (section 3.2.2)
 * and thick restart (section 3.3), every product by Algorithms 2/3.
 * Reorthogonalisation is classical Gram-Schmidt: in SSA_PREC_F64 the first
 * projection h = Q^T w; nothing more when max |h_i| <= 1e-12 ||w|| (w is
 * orthogonal to Q to that level already); otherwise the update fused with a
 * second projection, and that projection's update only when ||w'||^2 <
 * ||w||^2 / 2 afterwards (Kahan-Parlett).  In SSA_PREC_F32C one projection
 * and one update (the FP32 products' own error, ~1e-7 sigma_1, is far above
 * one pass's double-float orthogonality).
 * The series is held scaled by an exact power of two (max |f| in [1/2, 1)),
 * so any finite units work; sigma, residuals and products are returned in
 * the caller's units.
 * f: N doubles, or NULL to reuse the series given to ssa_set_series.
 * 1 <= k <= min(L, K).  On SSA_OK or SSA_ENOCONV *out holds a new
 * decomposition (free it with ssa_decomp_destroy).
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ENOCONV, SSA_ENUMERIC, SSA_ECUDA.
 */
int ssa_decompose(ssa_plan_t plan, const double* f, int k, ssa_decomp_t* out);

/* Decomposition facts: k, converged flag, thick restarts, X / X^T products applied, Krylov dimension d. */
int ssa_decomp_info(ssa_decomp_t d, int* k, int* converged, int* restarts, int64_t* matvecs, int* krylov_dim);

/*
 * Copy results out: sigma (k), U (L x k), V (K x k), resid (k; the
 * residual estimates |alpha_{c+1}| |P[r, i]| from relation (2)).  Any
 * output pointer may be NULL to skip it.
 */
int ssa_decomp_get(ssa_decomp_t d, double* sigma, double* U, double* V, double* resid);

/*
 * Grouping and diagonal averaging (sections 2.3-2.4) of a decomposition:
 * for group g the series of length N obtained by Hankelizing
 * sum_{i in I_g} sigma_i u_i v_i^T, computed as Algorithm 4 (FFT
 * convolution of u_i and v_i divided by the antidiagonal counts) summed in
 * the frequency domain.  Groups are CSR: members of group g are
 * grp_idx[grp_off[g] .. grp_off[g+1]-1], indices in [0, k), disjoint.
 * out: m x N (group g at out + g*N).
 * Errors: SSA_EINVAL (bad or overlapping groups), SSA_ECUDA.
 */
int ssa_reconstruct(ssa_decomp_t d, const int32_t* grp_off, const int32_t* grp_idx, int m, double* out);

/*
 * Algorithm 4 on caller-supplied triples: for each group the diagonal
 * average of sum_i sigma_i u_i v_i^T.  sigma (r), U (L x r, leading
 * dimension ldu >= L), V (K x r, ldv >= K); groups as in ssa_reconstruct
 * with indices in [0, r).  out: m x N.
 */
int ssa_hankelize(ssa_plan_t plan, const double* sigma, const double* U, int64_t ldu, const double* V, int64_t ldv,
                  int r, const int32_t* grp_off, const int32_t* grp_idx, int m, double* out);

/* ---- batched decompositions (many series in one launch) ----------------- */

typedef struct ssa_batch_s* ssa_batch_t;

/*
 * The truncated SVD of ssa_decompose for nseries independent series in one
 * persistent launch: each CTA of the GPU takes series from a device work
 * queue (largest first) and runs the whole method for that series inside
 * the CTA (spectrum, Algorithms 1-3 with CGS2 reorthogonalisation, thick
 * restart, projected SVD, Ritz vectors, sign rule).
 *   f:        all series back to back (host or device), series i is
 *             f[offsets[i] .. offsets[i+1]-1], offsets[0] = 0 (nseries + 1 int64)
 *   Ls, ks:   window and number of triples per series (nseries each)
 *   opts:     as for plans; opts->krylov_dim / keep apply to every series.
 * Limits: N <= 32768 (SSA_PREC_F32C) or N <= 16384 (SSA_PREC_F64); Krylov
 * dimension min(max(2k, k+32), min(L, K)) <= 72, so k <= 36 unless min(L, K) <= 72.
 * With opts->refine = SSA_REFINE_ON every series needs N <= 16384.
 * On SSA_OK or SSA_ENOCONV (some series not converged) *out holds the results.
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ENOCONV, SSA_ENUMERIC, SSA_ECUDA.
 */
int ssa_decompose_batch(int nseries, const double* f, const int64_t* offsets, const int64_t* Ls, const int32_t* ks,
                        const ssa_opts_t* opts, ssa_batch_t* out);

/* Facts of series i: k, converged flag, thick restarts, products applied. */
int ssa_batch_info(ssa_batch_t b, int i, int* k, int* converged, int* restarts, int64_t* matvecs);

/*
 * The same work split for repeated runs over series of unchanged sizes (a
 * bootstrap, a stream of equally shaped batches):
 *   ssa_batch_plan: validation, work order, twiddle tables, CTA slots and
 *     outputs, once (no series data; all device memory is allocated here);
 *   ssa_batch_run: one run on opts->stream for the series f (device memory,
 *     or host memory copied into the batch's own buffer; pinned host memory
 *     or device memory keeps the call capturable).  It only enqueues
 *     memsets and the persistent kernel(s): no allocation, no host copy of
 *     results and no synchronisation, so a CUDA graph can capture it;
 *   ssa_batch_wait: waits for the last run and returns its status as
 *     ssa_decompose_batch does.
 * ssa_batch_get / ssa_batch_info / ssa_batch_reconstruct read the results
 * of the last waited run.  Errors: as ssa_decompose_batch.
 */
int ssa_batch_plan(int nseries, const int64_t* offsets, const int64_t* Ls, const int32_t* ks, const ssa_opts_t* opts,
                   ssa_batch_t* out);
int ssa_batch_run(ssa_batch_t b, const double* f);
int ssa_batch_wait(ssa_batch_t b);

/* Results of series i: sigma (k), U (L x k), V (K x k), resid (k); NULL skips an output. */
int ssa_batch_get(ssa_batch_t b, int i, double* sigma, double* U, double* V, double* resid);

/*
 * Grouped Hankelization (Algorithm 4 summed over each group, divided by the
 * antidiagonal counts of section 5) of every series of a batch, with the
 * same groups for all series: CSR groups as in ssa_reconstruct, indices
 * below every series' k.  out: for series i, an m x N_i row-major block,
 * blocks in series order (sum_i m N_i doubles, host or device).
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_batch_reconstruct(ssa_batch_t b, const int32_t* grp_off, const int32_t* grp_idx, int m, double* out);

void ssa_batch_destroy(ssa_batch_t b);

/* ---- heterogeneity matrix (section 6.4) -------------------------------- */

/*
 * H-matrix G_{B,T}: g_ij = g(base_i, test_j) for the base subseries
 * base_i = (f_i, ..., f_{i+B-1}), i = 0..N-B, and the test subseries
 * test_j = (f_j, ..., f_{j+T-1}), j = 0..N-T, where g(F1, F2) is the
 * heterogeneity index (eq. g): the share of the squared norm of F2's
 * L-lagged vectors that lies outside the span of F1's left singular vectors
 * U_l, l in I.  (The paper prints F_{i,i+B}; the base holds B samples.)
 *   f:    N doubles (host or device)
 *   I:    nI distinct 1-based triple indices (host), each <= min(L, B-L+1)
 *   opts: precision, tolerance and stream of the base decompositions and products
 *   H:    (N-B+1) x (N-T+1) doubles, row-major (host or device), caller-owned
 * The base decompositions run as batched launches over the sliding windows
 * (one plan reused per window where B exceeds the batched engine's limits);
 * one Algorithm 3 product of the whole series per (base, l in I) gives
 * U_l^T X_t for every lagged vector X_t, and windowed sums of their squares
 * give every g_ij.  A test window that is identically zero gets g = 0.
 * Errors: SSA_EINVAL (need 1 < L < B <= N, L <= T <= N), SSA_ENOMEM,
 * SSA_ENOCONV (H is still written), SSA_ECUDA.
 */
int ssa_hmatrix(const double* f, int64_t N, int64_t L, int64_t B, int64_t T, const int32_t* I, int nI,
                const ssa_opts_t* opts, double* H);

/* ---- request server (continuous batching; not a step of the paper) ------ */

/*
 * A server decomposes series submitted at any time (ssa_decompose's truncated
 * SVD, Algorithms 1-3) while earlier requests are still running.  Requests are
 * admitted first-come-first-served as workers and the device-memory budget
 * free up.  Requests that fit the batched engine (ssa_decompose_batch limits)
 * are packed, as many as are queued (up to max_batch), into one persistent
 * launch; the others run the single-series path, several at once.  Every
 * worker has its own CUDA stream, so admitted requests overlap on the device.
 * Each request's spectrum and Lanczos state stay on the device until its
 * results are copied to host memory owned by the server.
 * Threads: all ssa_serve_* calls may be made from any host thread.
 */
typedef struct ssa_server_s* ssa_server_t;

typedef struct ssa_serve_opts {
  int precision;        /* SSA_PREC_F64 or SSA_PREC_F32C for every request (default SSA_PREC_F32C) */
  double tol;           /* as ssa_opts_t.tol (0 = the precision's default) */
  int64_t mem_budget;   /* device bytes that admitted requests may hold together (default 40 GiB) */
  int workers;          /* single-series requests running at once (default 8, at most 64).  Every worker
                           has its own stream, and CUDA maps streams onto 8 hardware work queues unless
                           CUDA_DEVICE_MAX_CONNECTIONS is raised before the process creates its CUDA
                           context: measured on the 2000 req/s mix, 16 workers with 32 connections
                           served 80 requests/s, 8 workers 77, 16 workers with 8 connections 71 */
  int batch_workers;    /* batched launches running at once (default 1, at most 16; 0 = never batch) */
  int max_batch;        /* requests per batched launch (default 128) */
  int64_t batch_max_n;  /* only series with N <= this are batched (0 = the engine's limit, -1 = none) */
  int grid_cap;         /* ssa_opts_t.grid_cap of every single-series request (default 0: the whole device;
                           measured on the serving workload, shares of 2 x SMs / workers CTAs lowered the
                           capacity from 75 to 66 requests/s with 8 workers) */
} ssa_serve_opts_t;

#define SSA_SERVE_VECTORS 1  /* ssa_serve_submit outputs flag: keep U and V (else sigma and residuals only) */

typedef struct ssa_serve_info {
  int status;           /* SSA_OK, SSA_ENOCONV or the error of this request */
  int converged, restarts;
  int64_t matvecs;
  int batched;          /* 1 if it ran in a batched launch */
  double t_submit, t_start, t_done;  /* seconds since ssa_serve_create */
} ssa_serve_info_t;

typedef struct ssa_serve_stats {
  int64_t submitted, completed, queued, running;
  int64_t mem_in_use, mem_peak;  /* admitted device bytes (estimates), now and at the peak */
  int64_t batches, batched_requests;
} ssa_serve_stats_t;

/* Defaults: SSA_PREC_F32C, tol 0, 40 GiB, 8 workers, 1 batch worker, max_batch 128, batch_max_n 0. */
void ssa_serve_default_opts(ssa_serve_opts_t* opts);
/* Start the worker threads.  opts may be NULL (defaults).  Errors: SSA_EINVAL, SSA_ENOMEM. */
int ssa_serve_create(const ssa_serve_opts_t* opts, ssa_server_t* out);
/*
 * Queue one request: f (N doubles, host memory, copied before returning),
 * window L and k triples; outputs = 0 or SSA_SERVE_VECTORS.  *id names it.
 * Errors: SSA_EINVAL (sizes as ssa_embed_plan / ssa_decompose), SSA_ENOMEM
 * (the request alone needs more than the memory budget).
 */
int ssa_serve_submit(ssa_server_t srv, const double* f, int64_t N, int64_t L, int k, int outputs, int64_t* id);
/* *done = 1 once request id has finished; waits up to timeout_s seconds (0 = do not wait). */
int ssa_serve_poll(ssa_server_t srv, int64_t id, double timeout_s, int* done);
/*
 * Copy a finished request's results to host buffers -- sigma (k), U (L x k),
 * V (K x k), resid (k), each may be NULL; U and V only if SSA_SERVE_VECTORS
 * was given -- fill *info (may be NULL) and release the request.  Returns
 * the request's status (SSA_OK, SSA_ENOCONV with results, or its error).
 */
int ssa_serve_take(ssa_server_t srv, int64_t id, double* sigma, double* U, double* V, double* resid,
                   ssa_serve_info_t* info);
int ssa_serve_stats(ssa_server_t srv, ssa_serve_stats_t* stats);
/* Finish the running requests, drop the queued ones and stop the threads. */
void ssa_serve_destroy(ssa_server_t srv);

/* ---- launch accounting (not part of the paper's method) ---------------- */

/*
 * Column tiling picked by the four-step autotuner for series of length N in
 * this precision: columns per CTA of the forward and inverse column passes
 * (0 when that size has not been planned yet in this process).  Plans with
 * M/2 above the single-CTA limit time the candidate tilings once per process
 * at ssa_embed_plan; every tiling gives bitwise the same results.
 */
int ssa_fft_tiling(int precision, int64_t N, int* cols_fwd, int* cols_inv);

/* Threads per CTA picked by the same autotuner for the forward column pass,
   the products' row pass and the inverse column pass (0 when not planned). */
int ssa_fft_threads(int precision, int64_t N, int* th_fwd, int* th_row, int* th_inv);

/* One entry per kernel of the library: launches, summed device time from
   CUDA events recorded around each launch, and the algorithmic bytes and
   flops charged to those launches (what the method must move / compute,
   e.g. one read of the basis for a projection). */
typedef struct ssa_kernel_stat {
  char name[32];
  uint64_t launches;
  double ms;
  double bytes;
  double flops;
} ssa_kernel_stat_t;

/* on = 1: reset the per-kernel statistics and start recording (a pair of
   CUDA events around every launch, on the launch's stream); on = 0: stop. */
int ssa_stats_enable(int on);

/* Synchronise the device, then copy up to max entries to out; *count gets
   the number of kernel entries available. */
int ssa_stats_get(ssa_kernel_stat_t* out, int max, int* count);

/* Total kernels launched by the library in this process. */
uint64_t ssa_kernel_launches(void);

/*
 * Host-side fault injection for tests of the error paths (not part of the
 * paper's method): with after >= 0, the next `after` device allocations made
 * by the single-series calls (ssa_embed_plan, ssa_set_series, ssa_matvec,
 * ssa_decompose, ssa_reconstruct, ssa_hankelize) succeed and the one after
 * them fails as if the device were out of memory (no allocator is called),
 * so that call returns SSA_ENOMEM; the injection then disarms itself.
 * after < 0 disarms it.  Nothing on the device is made to fail.
 */
int ssa_fault_inject_alloc(int64_t after);

/*
 * The ghost filter of SSA_REORTH_NONE on the host (no device access), exposed so that it can be
 * checked on its own (section 3.2.1, the Cullum-Willoughby test).  sigma: the c singular values of
 * the projected matrix B in descending order; sigma_hat: the c_hat singular values of B without its
 * first row; resid: the residual estimates of sigma's Ritz pairs.  Two values agree when they
 * differ by at most 1e-10 sigma[0]; values at or below that are not candidates.  Walking sigma's
 * groups of agreeing values in descending order, a group of one value that agrees with a sigma_hat
 * value is spurious; any other group keeps its member with the smallest residual.  keep (k
 * entries, caller-owned) receives the first k kept indices in ascending order, padded with the
 * largest unused indices when fewer pass; *converged = 1 when k passed and every kept residual is
 * <= tol sigma[0].  Errors: SSA_EINVAL (NULL pointer, k outside [1, c], sigma not descending,
 * non-finite input).
 */
int ssa_cw_filter(const double* sigma, int c, const double* sigma_hat, int c_hat, const double* resid, int k,
                  double tol, int32_t* keep, int* converged);

/* ---- allocation-free product (no counterpart in the paper) -------------- */

/*
 * ssa_matvec_noalloc -- y = X x (transpose = 0, x of length K, y of length L)
 * or y = X^T x (transpose = 1, x of length L, y of length K) for the series
 * f of length N, computing the spectrum of f and the product in one call
 * without allocating any device memory.
 *
 * For callers that cannot allocate: code running under a host framework that
 * owns all device memory through its own pool (a raw cudaMalloc there can
 * fail or fragment the pool), and latency-critical paths where cudaMalloc /
 * cudaFree, which may synchronise the device, are not acceptable.
 *
 * Its working memory (spectrum, FFT scratch, twiddle tables; about 1.3 MB)
 * is one file-scope __device__ array of fixed size that every GPU which loads
 * the library holds until the process exits.  Limits: N <= 65536; f, x and y
 * must be device pointers (host buffers would need staging); precision is
 * SSA_PREC_F64 or SSA_PREC_F32C.  Larger series or host buffers: use a plan
 * (ssa_embed_plan, ssa_set_series, ssa_matvec).
 *
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call
 * before any stream capture.  Work is enqueued on `stream` (a cudaStream_t,
 * NULL = default stream) and the call returns without synchronising.
 * Every call reuses the same array: each call writes everything it reads
 * (nothing needs to start at zero), so calls that overlap on the GPU -- on
 * different streams, or from different threads -- race and must be ordered
 * by the caller.
 * Errors: SSA_EINVAL (NULL or host pointer, sizes, N > 65536), SSA_ECUDA.
 */
int ssa_matvec_noalloc(const double* f, int64_t N, int64_t L, int transpose, const double* x, double* y,
                       int precision, void* stream);

/* Destroy decompositions before the plan they came from (their memory is
 * released in the order of the plan's stream). */
void ssa_plan_destroy(ssa_plan_t plan);
void ssa_decomp_destroy(ssa_decomp_t d);
const char* ssa_strerror(int code);
const char* ssa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SSA_GB300_H */
