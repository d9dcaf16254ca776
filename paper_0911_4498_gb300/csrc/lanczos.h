// Host-side interface of the Lanczos engine kernels (lanczos_kernels.cu).
#pragma once
#include "common.cuh"

namespace ssa {

constexpr int RT = 256;              // threads per reorthogonalisation block
constexpr int RP = 4;                // row pairs per thread
constexpr int SLAB = 2 * RT * RP;    // rows per block
constexpr int MAXCOL = 512;          // largest basis size (Krylov dimension + 1)
constexpr int SVD_THREADS = 1024;
constexpr int PRE_THREADS = 1024;
constexpr int PRE_SMEM_MAX = 200 * 1024;  // FP32 preconditioning of the projected SVD when r*c + c*c floats fit
constexpr int PRE_SWEEPS = 12;          // FP32 preconditioner sweeps at most
constexpr int SVD_STAGE_MAX = 200 * 1024;  // shared memory for the df64 Jacobi (A and W staged when they fit)
constexpr int SVD_CL = 8;                  // CTAs of the clustered projected-SVD kernel (portable cluster size)
constexpr int SVD_CL_THREADS = 512;        // threads per CTA of that kernel
constexpr int FUSED_MAXCOL = 200;   // largest basis for the fused update+projection pass
// Skip test of the gated reorthogonalisation (when enabled with a level tau):
// with h = Q^T w from the first projection and w' = w - h_l q_l (l the newest
// column), the update and the second projection are skipped when
// max_{i<l} |h_i| <= tau ||w'|| and ||w||^2 <= SKIP_RATIO ||w'||^2 (w' is then
// orthogonal to Q to that level).
constexpr double SKIP_RATIO = 1e4;

struct ReorthWork {
  df64* part;    // [blocks][ldp] partial sums (row tiles of SLAB rows)
  df64* part2;   // [tiles][ldp] partial sums of the fused pass (tiles of 64 rows)
  int ldp;
  int ldp2;      // leading dimension of part2 (FUSED_MAXCOL + 1)
  df64* h;       // projection coefficients of the first pass; h[ncols] = ||w||^2 (MAXCOL + 1)
  df64* h2;      // the same for the second pass; h2[ncols] = ||w'||^2 (MAXCOL + 1)
  int* gate;     // 1 when the third pass must run (Kahan-Parlett test on the device)
  int* run;      // 1 when the second pass must run (skip test on the device)
  int* skip;     // 1 when the skip test fired (then *run == 0 and *gate == 0)
  double skip_tau;  // level of the skip test in REORTH_GATED (0: no skip test)
  int grid_cap = 0;  // most blocks of the persistent passes and the cooperative kernels (0: no cap)
  // set by launch_cgs2 for launch_normalize_coop: when *skip_flag is 1 on the
  // device, the normalisation forms w <- w - h[ncols-1] q_{ncols-1} and its
  // norm itself (h = the first projection, in h)
  const int* skip_flag;
  df64* nrm;     // squared norm after the last update (see nrm_blocks)
  // launch_cgs2 may leave the final squared norm as per-block partial sums,
  // column nrm_col of the first nrm_blocks rows of part2, for the following
  // launch_normalize_coop to add up; nrm_blocks == 0, or *nrm_gate == 0 on the
  // device, means *nrm holds it
  int nrm_blocks;
  int nrm_col;
  const int* nrm_gate;
  int* counter;  // last-block counter (returns to 0 after each kernel)
  df64* coop;    // [coop_blocks()][MAXCOL + 1] scratch of the breakdown branch
  unsigned* status;  // device status word (SSA_DEV_* bits)
};

struct SvdWork {
  df64 *A, *W;            // Jacobi work: r x c and c x c (column-major)
  df64 *sigma, *P, *Q;    // sorted outputs
  double *resid, *sigma_d;
  int* conv;
  int max_sweeps;
  float rot_tol;
};

// Partial reorthogonalisation state: estimates of u_i.u_j (M) and v_i.v_j (N),
// FP32, lde x lde each; eps is the relative error level of the products; force
// holds the "reorthogonalise the next step too" flags of the two sides.
struct ProState {
  float* M;
  float* N;
  int lde;
  float eps;
  int* force;
};

int reorth_blocks(int64_t dim);
int fused_tiles(int64_t dim);
void reorth_setup();
// Classical Gram-Schmidt of w against the ncols columns of Q, then the squared
// norm ||w||^2 for the next launch_normalize_coop (in *rw.nrm, or as partial
// sums that it adds up).  REORTH_ONCE: one projection and update (two passes over
// Q).  REORTH_GATED: the first projection h = Q^T w; if rw.skip_tau > 0 and the
// skip test holds (skip_tau, SKIP_RATIO) only w - h_l q_l remains to form, which the
// normalisation does; otherwise the update fused with a second projection,
// and that projection's update (a third pass) only when ||w'||^2 < ||w||^2 / 2
// after the first (Kahan-Parlett), so the result is orthogonal to Q to
// working precision.  Bases wider than FUSED_MAXCOL always take two full rounds.
// REORTH_PRO: the passes of REORTH_GATED, all gated by rw.run (set by launch_pro_pre).
enum { REORTH_ONCE = 1, REORTH_GATED = 2, REORTH_PRO = 3 };
void launch_cgs2(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, ReorthWork& rw, int mode,
                 cudaStream_t s);
int coop_blocks();
int launch_normalize_coop(df64* w, int64_t dim, ReorthWork& rw, df64* qcol, df64* bentry, df64* est,
                          const df64* Q, int64_t ldq, int ncols, uint64_t seed, uint64_t stream, unsigned* status,
                          cudaStream_t s);
// PRO pre-step (cooperative): w -= coef * qprev (if qprev), the new vector's orthogonality
// estimates and the decision in *rw.run (else *rw.gate = 0, *rw.nrm = ||w||^2); side 0: new u
// (index newidx) from v_src, side 1: new v from u_src; prev: the coupled vector, -1 if none
int launch_pro_pre(df64* w, int64_t dim, const df64* qprev, const df64* coef, ReorthWork& rw, ProState& ps,
                   const df64* B, int ldb, int side, int newidx, int src, int cnt_same, int cnt_other, int prev,
                   const df64* est, cudaStream_t s);
void launch_pro_reset(ProState& ps, cudaStream_t s);
void launch_random_fill(df64* w, int64_t dim, uint64_t seed, uint64_t stream, cudaStream_t s);
void launch_small_svd(const df64* B, int ldb, int r, int c, SvdWork& sw, int k, double tol_conv,
                      df64* est, unsigned* status, cudaStream_t s);
void launch_restart_B(df64* B, int ldb, int nrows_clear, const SvdWork& sw, int r, int kk, int c_old,
                      cudaStream_t s);
void launch_ritz(const df64* Q, int64_t ldq, int r, const df64* P, int ldp, int ncol, df64* out, int64_t ldo,
                 int64_t dim, cudaStream_t s);
void launch_copy_df(const df64* src, df64* dst, int64_t n, cudaStream_t s);
// Q[:, j] /= ||Q[:, j]||, j < ncol (one block per column)
void launch_normalize_cols(df64* Q, int64_t ldq, int64_t dim, int ncol, cudaStream_t s);
void launch_sign(const df64* U, int64_t ldu, int64_t dim, int k, int* sgn, cudaStream_t s);
void launch_store_cols(const df64* src, int64_t lds, int64_t dim, int ncol, const int* sgn, double* dst, int64_t ldd,
                       cudaStream_t s);
void launch_df_to_double(const df64* src, double* dst, int64_t n, cudaStream_t s);
// out[j] = sum_i A[j*lda + i] * B[j*ldb + i] over i < dim, in FP64 (one block per column)
void launch_col_dots(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t dim, int ncol, double* out,
                     cudaStream_t s);
void launch_double_to_df(const double* src, int64_t lds, df64* dst, int64_t ldd, int64_t dim, int ncol,
                         cudaStream_t s);

}  // namespace ssa
