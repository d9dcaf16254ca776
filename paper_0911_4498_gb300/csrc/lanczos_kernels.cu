// Device kernels of the Golub-Kahan-Lanczos engine (section 3) other than the
// reorthogonalisation passes (cgs.cu): the normalisation with breakdown
// replacement, the SVD of the projected matrix B by one-sided Jacobi (one CTA,
// or an 8-CTA cluster), the Ritz-vector products U P and V Q of a thick
// restart, and the output conversion with the sign rule.  All vectors and the
// projected problem are double-float (df64).
#include <cooperative_groups.h>
#include <mutex>
#include "lanczos.h"
#include "lanczos_dev.cuh"
#include "prof.h"

namespace ssa {

__global__ void k_random_fill(df64* w, int64_t dim, uint64_t seed, uint64_t stream) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = sm64_uniform_pm1(seed, stream, i);
}

namespace cg = cooperative_groups;

// Normalise w into qcol and record the coupling coefficient (one cooperative
// launch).  ||w||^2 is *nrm2 or, when the reorthogonalisation left it as
// per-block partial sums, their sum.  Usual case: beta = ||w|| > 1e-14 * est,
// qcol = w / beta.
// Breakdown (beta at or below that level, including 0): the coefficient is
// recorded as 0 and w is replaced by a seeded random vector, orthogonalised
// against the ncols basis columns by CGS2 inside the kernel (grid-wide
// barriers between the passes); if it vanishes the basis already spans the
// space and qcol is set to zero.  est (largest coupling / singular value
// seen) is raised by block 0 at the end; other blocks may read the old or
// the new value, which gives the same decision because the new value is beta.
__global__ void __launch_bounds__(256) k_normalize_coop(df64* __restrict__ w, int64_t dim,
                                                        const df64* __restrict__ nrm2, df64* __restrict__ qcol,
                                                        df64* __restrict__ bentry, df64* est,
                                                        const df64* __restrict__ Q, int64_t ldq, int ncols,
                                                        df64* __restrict__ scratch, int lds, uint64_t seed,
                                                        uint64_t stream, unsigned* status,
                                                        const df64* __restrict__ npart, int nblk, int ldnp,
                                                        int ncol, const int* ngate, const int* skipf,
                                                        const df64* __restrict__ hproj) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  __shared__ df64 sh[32];
  __shared__ df64 hs[MAXCOL + 4];
  if (skipf && *skipf) {
    // the reorthogonalisation's skip test fired: w <- w - h_l q_l (l = ncols - 1, h_l from
    // its first projection) and ||w||^2 here, summed over the grid in block order
    cg::grid_group grid = cg::this_grid();
    const df64 hl = hproj[ncols - 1];
    const df64* ql = Q + (int64_t)(ncols - 1) * ldq;
    df64 a = df_zero();
    for (int64_t i = tid; i < dim; i += stride) {
      const df64 x = df_sub(w[i], df_mul(hl, ql[i]));
      w[i] = x;
      a = df_fma(x, x, a);
    }
    a = block_sum_df(a, sh);
    if (threadIdx.x == 0) scratch[(int64_t)blockIdx.x * lds + MAXCOL] = a;
    grid.sync();
    if (threadIdx.x < 32) {  // lane-strided over the blocks, then a warp butterfly (same sum in every block)
      df64 t = df_zero();
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t = df_add(t, scratch[(int64_t)b * lds + MAXCOL]);
      t = warp_sum_df(t);
      if (threadIdx.x == 0) sh[0] = t;
    }
  } else if (threadIdx.x < 32) {
    // ||w||^2: *nrm2, or the sum of the reorthogonalisation's per-block partials (npart[b][ncol],
    // b < nblk; lane-strided then a warp butterfly, the same value in every block)
    df64 v;
    if (nblk > 0 && !(ngate && *ngate == 0)) {
      df64 a = df_zero();
      for (int b = threadIdx.x; b < nblk; b += 32) a = df_add(a, npart[(int64_t)b * ldnp + ncol]);
      v = warp_sum_df(a);
    } else {
      v = *nrm2;
    }
    if (threadIdx.x == 0) sh[0] = v;
  }
  __syncthreads();
  const df64 beta = df_sqrt(sh[0]);
  __syncthreads();  // sh is reused below
  if (!isfinite(beta.hi) && tid == 0) atomicOr(status, SSA_DEV_NONFINITE);
  const float thr = 1e-14f * est->hi;
  if (beta.hi > thr && beta.hi > 0.f && isfinite(beta.hi)) {
    const df64 inv = df_div(make_df(1.f, 0.f), beta);
    for (int64_t i = tid; i < dim; i += stride) qcol[i] = df_mul(w[i], inv);
    if (tid == 0) {
      *bentry = beta;
      if (df_gt(beta, *est)) *est = beta;
    }
    return;
  }
  // ---- breakdown: the whole grid takes this branch
  cg::grid_group grid = cg::this_grid();
  if (tid == 0) {
    *bentry = df_zero();
    atomicOr(status, SSA_DEV_BREAKDOWN);
  }
  for (int64_t i = tid; i < dim; i += stride) w[i] = sm64_uniform_pm1(seed, stream, i);
  for (int pass = 0; pass < 2 && ncols > 0; ++pass) {
    grid.sync();
    for (int c = 0; c < ncols; ++c) {
      const df64* q = Q + (int64_t)c * ldq;
      df64 a = df_zero();
      for (int64_t i = tid; i < dim; i += stride) a = df_fma(q[i], w[i], a);
      a = block_sum_df(a, sh);
      if (threadIdx.x == 0) scratch[(int64_t)blockIdx.x * lds + c] = a;
    }
    grid.sync();
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
      df64 a = df_zero();
      for (int b = 0; b < (int)gridDim.x; ++b) a = df_add(a, scratch[(int64_t)b * lds + c]);
      hs[c] = a;
    }
    __syncthreads();
    for (int64_t i = tid; i < dim; i += stride) {
      df64 a = df_zero();
      for (int c = 0; c < ncols; ++c) a = df_fma(Q[(int64_t)c * ldq + i], hs[c], a);
      w[i] = df_sub(w[i], a);
    }
  }
  grid.sync();
  df64 a = df_zero();
  for (int64_t i = tid; i < dim; i += stride) a = df_fma(w[i], w[i], a);
  a = block_sum_df(a, sh);
  if (threadIdx.x == 0) scratch[(int64_t)blockIdx.x * lds + MAXCOL] = a;
  grid.sync();
  if (threadIdx.x == 0) {
    df64 t = df_zero();
    for (int b = 0; b < (int)gridDim.x; ++b) t = df_add(t, scratch[(int64_t)b * lds + MAXCOL]);
    sh[0] = t;
  }
  __syncthreads();
  const df64 nb = df_sqrt(sh[0]);
  // the random vector had norm ~ sqrt(dim/3) before orthogonalisation
  const bool alive = nb.hi > 1e-6f * sqrtf((float)dim / 3.f);
  const df64 inv = alive ? df_div(make_df(1.f, 0.f), nb) : df_zero();
  for (int64_t i = tid; i < dim; i += stride) qcol[i] = df_mul(w[i], inv);
}


// ---------------------------------------------------------------- partial reorthogonalisation
// PRO pre-step of a half-step (cooperative).  All blocks: w <- w - coef q_prev
// (the one known coupling of the bidiagonalisation, when there is one) and
// ||w||^2 summed over the grid.  Block 0 then updates the orthogonality
// estimates of the new vector against the older ones of its side, from the
// projected matrix B (X v_b = sum_a B[a][b] u_a, X^T u_a = sum_b B[a][b] v_b):
//   new u from v_s, coupling u_p:  u_i.w = sum_b B[i][b] N[s][b] - B[p][s] M[p][i]
//   new v from u_s, coupling v_p:  v_i.w = sum_a B[a][i] M[s][a] - B[s][p] N[p][i]
// each plus a rounding term eps ||X|| with the sign of the sum, divided by
// ||w|| (estimates in FP32: only their magnitude matters).  The Gram-Schmidt
// passes run (*run = 1) when an estimate exceeds sqrt(eps), when the caller
// forces it, or on the step after one that ran (the estimates of a vector
// built on a reorthogonalised one are not yet small); then the new vector's
// estimates are reset to eps.  Otherwise *gate = 0 and *nrm = ||w||^2 for the
// normalisation.
struct ProArgs {
  df64* w;
  int64_t dim;
  const df64* qprev;
  const df64* coef;
  df64* nrm;
  int* run;
  int* gate;
  float* M;  // [u][u] estimates, leading dimension lde
  float* N;  // [v][v]
  int lde;
  const df64* B;
  int ldb;
  int side;    // 0: new u, 1: new v
  int newidx;  // index of the new vector on its side
  int src;     // index of the product's input vector (other side)
  int cnt_same, cnt_other;  // vectors on the new vector's side / the other side before the new one
  int prev;    // index of the coupled vector on the same side, -1 if none
  float eps;
  const df64* est;
  int* force;  // [0] u side, [1] v side
  df64* scratch;
  int lds;
};

__global__ void __launch_bounds__(256) k_pro_pre(ProArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ df64 sh[32];
  __shared__ float fm[32];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const df64 c = a.coef ? *a.coef : df_zero();
  df64 acc = df_zero();
  for (int64_t i = tid; i < a.dim; i += stride) {
    df64 x = a.w[i];
    if (a.qprev) x = df_sub(x, df_mul(c, a.qprev[i]));
    a.w[i] = x;
    acc = df_fma(x, x, acc);
  }
  acc = block_sum_df(acc, sh);
  if (threadIdx.x == 0) a.scratch[(int64_t)blockIdx.x * a.lds + MAXCOL] = acc;
  grid.sync();
  if (blockIdx.x != 0) return;
  if (threadIdx.x < 32) {
    df64 t = df_zero();
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t = df_add(t, a.scratch[(int64_t)b * a.lds + MAXCOL]);
    t = warp_sum_df(t);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  const df64 n2 = sh[0];
  const float nw = sqrtf(fmaxf(n2.hi, 0.f));
  const float tolr = a.eps * a.est->hi;
  float* E = (a.side == 0 ? a.M : a.N) + (int64_t)a.newidx * a.lde;
  const float* Eo = (a.side == 0 ? a.N : a.M) + (int64_t)a.src * a.lde;   // estimates of the source vector
  const float* Ep = a.prev >= 0 ? (a.side == 0 ? a.M : a.N) + (int64_t)a.prev * a.lde : nullptr;
  const float cpl = a.prev >= 0 ? (a.side == 0 ? a.B[(int64_t)a.prev * a.ldb + a.src].hi
                                                : a.B[(int64_t)a.src * a.ldb + a.prev].hi)
                                 : 0.f;
  // one warp per estimate, its lanes over the other side's vectors
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  float m = 0.f;
  for (int i = threadIdx.x >> 5; i < a.cnt_same; i += nwarp) {
    float s = 0.f;
    if (i != a.prev) {
      if (a.side == 0)
        for (int b = lane; b < a.cnt_other; b += 32) s = fmaf(a.B[(int64_t)i * a.ldb + b].hi, Eo[b], s);
      else
        for (int b = lane; b < a.cnt_other; b += 32) s = fmaf(a.B[(int64_t)b * a.ldb + i].hi, Eo[b], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (i != a.prev && Ep) s = fmaf(-cpl, Ep[i], s);
    const float v = nw > 0.f ? (s + copysignf(tolr, s)) / nw : 1.f;
    if (lane == 0) E[i] = v;
    m = fmaxf(m, fabsf(v));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) fm[threadIdx.x >> 5] = m;
  __syncthreads();
  __shared__ int s_run;
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, fm[i]);
    const int f = a.force[a.side];
    const int run = f || !(m <= sqrtf(a.eps)) ? 1 : 0;
    a.force[a.side] = (run && !f) ? 1 : 0;
    *a.run = run;
    if (!run) {
      *a.gate = 0;
      *a.nrm = n2;
    }
    s_run = run;
  }
  __syncthreads();
  if (s_run)
    for (int i = threadIdx.x; i < a.cnt_same; i += blockDim.x) E[i] = a.eps;
  if (threadIdx.x == 0) E[a.newidx] = 1.f;
}

// estimates of a fresh basis (after a restart, or at the start): eps off the diagonal, 1 on it
__global__ void k_pro_reset(float* M, float* N, int lde, int n, float eps, int* force) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * lde; e += gridDim.x * blockDim.x) {
    const int i = e / lde, j = e - i * lde;
    const float v = i == j ? 1.f : eps;
    M[e] = v;
    N[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x < 2) force[threadIdx.x] = 0;
}

// ---------------------------------------------------------------- projected SVD
// One-CTA projected SVD (see svd_jacobi_body / svd_precondition_body).
__global__ void __launch_bounds__(SVD_THREADS) k_small_svd(const df64* __restrict__ B, int ldb, int r, int c,
                                                           df64* __restrict__ A, df64* __restrict__ W, int cc,
                                                           df64* __restrict__ sigma, df64* __restrict__ P,
                                                           df64* __restrict__ Qv, double* __restrict__ resid,
                                                           double* __restrict__ sigma_d, int k, double tol_conv,
                                                           int* conv, df64* est, unsigned* status, int max_sweeps,
                                                           float rot_tol, int warm, int staged) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  svd_jacobi_body<SVD_THREADS>(B, ldb, r, c, A, W, cc, sigma, P, Qv, resid, sigma_d, k, tol_conv, conv, est, status,
                               max_sweeps, rot_tol, warm, staged ? reinterpret_cast<df64*>(smem_raw) : nullptr);
}

// One-sided Jacobi of the projected matrix on a cluster of SVD_CL CTAs: the
// columns of A (r each) and W (c each) live in the CTAs' shared memory,
// column j in CTA j % SVD_CL (distributed shared memory); each rotation pair
// of a round is one warp anywhere in the cluster, and the hardware cluster
// barrier separates the rounds.  The arithmetic of every pair is that of
// svd_jacobi_body (same order, same reductions), so the results are the
// same bit for bit; the work of a round is spread over SVD_CL SMs instead of
// one.
template <int NPL>
__global__ void __cluster_dims__(SVD_CL, 1, 1) __launch_bounds__(SVD_CL_THREADS)
    k_small_svd_cluster(const df64* __restrict__ B, int ldb, int r, int c, const df64* __restrict__ Ain,
                        const df64* __restrict__ Win, int cc, df64* __restrict__ sigma, df64* __restrict__ P,
                        df64* __restrict__ Qv, double* __restrict__ resid, double* __restrict__ sigma_d, int k,
                        double tol_conv, int* conv, df64* est, unsigned* status, int max_sweeps, float rot_tol,
                        int warm) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nloc = (c + SVD_CL - 1) / SVD_CL;
  df64* Aloc = reinterpret_cast<df64*>(smem_raw);
  df64* Wloc = Aloc + (size_t)nloc * r;
  df64* nrm_loc = Wloc + (size_t)nloc * c;
  __shared__ int rotated_s;
  __shared__ float maxr_s;
  __shared__ int ok_s;
  const int lane = threadIdx.x & 31, nwl = SVD_CL_THREADS / 32;
  const int gwarp = rank * nwl + (threadIdx.x >> 5), nwarps = SVD_CL * nwl;
  auto colA = [&](int j) { return cl.map_shared_rank(Aloc + (size_t)(j / SVD_CL) * r, j % SVD_CL); };
  auto colW = [&](int j) { return cl.map_shared_rank(Wloc + (size_t)(j / SVD_CL) * c, j % SVD_CL); };
  for (int jl = 0; jl < nloc; ++jl) {
    const int j = jl * SVD_CL + rank;
    if (j >= c) break;
    for (int i = threadIdx.x; i < r; i += SVD_CL_THREADS)
      Aloc[(size_t)jl * r + i] = warm ? Ain[(size_t)j * r + i] : B[(size_t)i * ldb + j];
    for (int i = threadIdx.x; i < c; i += SVD_CL_THREADS)
      Wloc[(size_t)jl * c + i] = warm ? Win[(size_t)j * c + i] : make_df(i == j ? 1.f : 0.f, 0.f);
  }
  cl.sync();
  int sweeps_used = -1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      rotated_s = 0;
      maxr_s = 0.f;
    }
    __syncthreads();
    for (int rnd = 0; rnd < cc - 1; ++rnd) {
      for (int pr = gwarp; pr < cc / 2; pr += nwarps) {
        const int2 pq = rr_pair(rnd, pr, cc);
        const int p = pq.x, q = pq.y;
        if (p >= c || q >= c) continue;
        df64* ap = colA(p);
        df64* aq = colA(q);
        df64* wp = colW(p);
        df64* wq = colW(q);
        df64 al = df_zero(), be = df_zero(), ga = df_zero();
        // NPL > 0: the lane's pieces of both columns of A and W in registers, loaded at once
        df64 xa[NPL > 0 ? NPL : 1], ya[NPL > 0 ? NPL : 1], xw[NPL > 0 ? NPL : 1], yw[NPL > 0 ? NPL : 1];
        if constexpr (NPL > 0) {
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            const int i = lane + 32 * u;
            xa[u] = i < r ? ap[i] : df_zero();
            ya[u] = i < r ? aq[i] : df_zero();
            xw[u] = i < c ? wp[i] : df_zero();
            yw[u] = i < c ? wq[i] : df_zero();
          }
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            if (lane + 32 * u < r) {
              al = df_fma(xa[u], xa[u], al);
              be = df_fma(ya[u], ya[u], be);
              ga = df_fma(xa[u], ya[u], ga);
            }
          }
        } else {
          for (int i = lane; i < r; i += 32) {
            const df64 x = ap[i], y = aq[i];
            al = df_fma(x, x, al);
            be = df_fma(y, y, be);
            ga = df_fma(x, y, ga);
          }
        }
        al = warp_sum_df(al);
        be = warp_sum_df(be);
        ga = warp_sum_df(ga);
        if (!(al.hi > 0.f) || !(be.hi > 0.f)) continue;
        const df64 nab = df_mul(df_sqrt(al), df_sqrt(be));
        const df64 thr = df_mul_f(nab, rot_tol);
        if (!df_gt(df_abs(ga), thr)) continue;
        if (lane == 0) {
          const float ratio = fabsf(ga.hi) / nab.hi;
          atomicMax(reinterpret_cast<int*>(&maxr_s), __float_as_int(ratio));
        }
        const df64 zeta = df_div(df_sub(be, al), df_scale(ga, 2.f));
        const df64 az = df_abs(zeta);
        df64 t;
        if (az.hi > 1e15f) {
          t = df_div(make_df(1.f, 0.f), df_scale(zeta, 2.f));
        } else {
          t = df_div(make_df(zeta.hi >= 0.f ? 1.f : -1.f, 0.f),
                     df_add(az, df_sqrt(df_add(make_df(1.f, 0.f), df_mul(zeta, zeta)))));
        }
        const df64 cs = df_div(make_df(1.f, 0.f), df_sqrt(df_add(make_df(1.f, 0.f), df_mul(t, t))));
        const df64 sn = df_mul(cs, t);
        if constexpr (NPL > 0) {
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            const int i = lane + 32 * u;
            if (i < r) {
              ap[i] = df_sub(df_mul(cs, xa[u]), df_mul(sn, ya[u]));
              aq[i] = df_add(df_mul(sn, xa[u]), df_mul(cs, ya[u]));
            }
            if (i < c) {
              wp[i] = df_sub(df_mul(cs, xw[u]), df_mul(sn, yw[u]));
              wq[i] = df_add(df_mul(sn, xw[u]), df_mul(cs, yw[u]));
            }
          }
        } else {
          for (int i = lane; i < r; i += 32) {
            const df64 x = ap[i], y = aq[i];
            ap[i] = df_sub(df_mul(cs, x), df_mul(sn, y));
            aq[i] = df_add(df_mul(sn, x), df_mul(cs, y));
          }
          for (int i = lane; i < c; i += 32) {
            const df64 x = wp[i], y = wq[i];
            wp[i] = df_sub(df_mul(cs, x), df_mul(sn, y));
            wq[i] = df_add(df_mul(sn, x), df_mul(cs, y));
          }
        }
        if (lane == 0) rotated_s = 1;
      }
      cl.sync();
    }
    int any = 0;
    float mr = 0.f;
    for (int qr = 0; qr < SVD_CL; ++qr) {
      any |= *cl.map_shared_rank(&rotated_s, qr);
      mr = fmaxf(mr, *cl.map_shared_rank(&maxr_s, qr));
    }
    cl.sync();  // every CTA has read the flags before they are reset
    if (!any || mr < 1e-10f) {
      sweeps_used = sweep + 1;
      break;
    }
  }
  if (rank == 0 && threadIdx.x == 0 && sweeps_used < 0) atomicOr(status, SSA_DEV_JACOBI_NOCONV);
  // column norms of the local columns
  for (int jl = threadIdx.x >> 5; jl < nloc; jl += nwl) {
    const int j = jl * SVD_CL + rank;
    if (j >= c) break;
    df64 sq = df_zero();
    for (int i = lane; i < r; i += 32) sq = df_fma(Aloc[(size_t)jl * r + i], Aloc[(size_t)jl * r + i], sq);
    sq = warp_sum_df(sq);
    if (lane == 0) nrm_loc[jl] = df_sqrt(sq);
  }
  cl.sync();
  // rank by descending sigma (ties: lower index first); the owner scatters its columns
  for (int jl = threadIdx.x >> 5; jl < nloc; jl += nwl) {
    const int j = jl * SVD_CL + rank;
    if (j >= c) break;
    const df64 sj = nrm_loc[jl];
    int rk = 0;
    for (int i = lane; i < c; i += 32) {
      const df64 si = *cl.map_shared_rank(nrm_loc + i / SVD_CL, i % SVD_CL);
      if (df_gt(si, sj) || (si.hi == sj.hi && si.lo == sj.lo && i < j)) ++rk;
    }
    for (int m = 16; m; m >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, m);
    const df64 inv = sj.hi > 0.f ? df_div(make_df(1.f, 0.f), sj) : df_zero();
    for (int i = lane; i < r; i += 32) P[(size_t)rk * r + i] = df_mul(Aloc[(size_t)jl * r + i], inv);
    for (int i = lane; i < c; i += 32) Qv[(size_t)rk * c + i] = Wloc[(size_t)jl * c + i];
    if (lane == 0) {
      sigma[rk] = sj;
      sigma_d[rk] = df_to_double(sj);
    }
  }
  cl.sync();
  if (rank != 0) return;
  // residuals from relation (2) and the convergence test
  const df64 alpha_res = B[(int64_t)(r - 1) * ldb + c];
  if (threadIdx.x == 0) ok_s = 1;
  __syncthreads();
  const double s1 = sigma_d[0];
  for (int m = threadIdx.x; m < c; m += SVD_CL_THREADS) {
    const double rm = fabs(df_to_double(df_mul(alpha_res, P[(int64_t)m * r + (r - 1)])));
    resid[m] = rm;
    if (m < k && !(rm <= tol_conv * s1)) ok_s = 0;
    if (!isfinite(rm)) atomicOr(status, SSA_DEV_NONFINITE);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *conv = ok_s;
    if (df_gt(sigma[0], *est)) *est = sigma[0];
  }
}

// The FP32 preconditioner of the projected SVD on an 8-CTA cluster: FP32
// one-sided Jacobi with the columns of A32 and W32 spread over the CTAs'
// shared memory (as k_small_svd_cluster), then the two Newton-Schulz steps
// and A = B W with their entries split over the cluster's threads.  Same
// arithmetic per entry as svd_precondition_body.
template <int NPL>
__global__ void __cluster_dims__(SVD_CL, 1, 1) __launch_bounds__(SVD_CL_THREADS)
    k_svd_precondition_cluster(const df64* __restrict__ B, int ldb, int r, int c, df64* __restrict__ A,
                               df64* __restrict__ W, df64* __restrict__ T1, int cc, int max_sweeps, float tol32) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nloc = (c + SVD_CL - 1) / SVD_CL;
  float* A32 = reinterpret_cast<float*>(smem_raw);
  float* W32 = A32 + (size_t)nloc * r;
  __shared__ int rotated_s;
  const int lane = threadIdx.x & 31, nwl = SVD_CL_THREADS / 32;
  const int gwarp = rank * nwl + (threadIdx.x >> 5), nwarps = SVD_CL * nwl;
  const int gtid = rank * SVD_CL_THREADS + threadIdx.x, gthreads = SVD_CL * SVD_CL_THREADS;
  auto colA = [&](int j) { return cl.map_shared_rank(A32 + (size_t)(j / SVD_CL) * r, j % SVD_CL); };
  auto colW = [&](int j) { return cl.map_shared_rank(W32 + (size_t)(j / SVD_CL) * c, j % SVD_CL); };
  for (int jl = 0; jl < nloc; ++jl) {
    const int j = jl * SVD_CL + rank;
    if (j >= c) break;
    for (int i = threadIdx.x; i < r; i += SVD_CL_THREADS) {
      const df64 b = B[(int64_t)i * ldb + j];
      A32[(size_t)jl * r + i] = b.hi + b.lo;
    }
    for (int i = threadIdx.x; i < c; i += SVD_CL_THREADS) W32[(size_t)jl * c + i] = i == j ? 1.f : 0.f;
  }
  cl.sync();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated_s = 0;
    __syncthreads();
    for (int rnd = 0; rnd < cc - 1; ++rnd) {
      for (int pr = gwarp; pr < cc / 2; pr += nwarps) {
        const int2 pq = rr_pair(rnd, pr, cc);
        const int p = pq.x, q = pq.y;
        if (p >= c || q >= c) continue;
        float* ap = colA(p);
        float* aq = colA(q);
        float* wp = colW(p);
        float* wq = colW(q);
        float al = 0.f, be = 0.f, ga = 0.f;
        float xa[NPL > 0 ? NPL : 1], ya[NPL > 0 ? NPL : 1], xw[NPL > 0 ? NPL : 1], yw[NPL > 0 ? NPL : 1];
        if constexpr (NPL > 0) {
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            const int i = lane + 32 * u;
            xa[u] = i < r ? ap[i] : 0.f;
            ya[u] = i < r ? aq[i] : 0.f;
            xw[u] = i < c ? wp[i] : 0.f;
            yw[u] = i < c ? wq[i] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            if (lane + 32 * u < r) {
              al = fmaf(xa[u], xa[u], al);
              be = fmaf(ya[u], ya[u], be);
              ga = fmaf(xa[u], ya[u], ga);
            }
          }
        } else {
          for (int i = lane; i < r; i += 32) {
            const float x = ap[i], y = aq[i];
            al = fmaf(x, x, al);
            be = fmaf(y, y, be);
            ga = fmaf(x, y, ga);
          }
        }
#pragma unroll
        for (int m = 16; m; m >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, m);
          be += __shfl_xor_sync(0xffffffffu, be, m);
          ga += __shfl_xor_sync(0xffffffffu, ga, m);
        }
        if (!(al > 0.f) || !(be > 0.f)) continue;
        if (!(fabsf(ga) > tol32 * sqrtf(al) * sqrtf(be))) continue;
        const float zeta = (be - al) / (2.f * ga);
        const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float cs = 1.f / sqrtf(1.f + t * t);
        const float sn = cs * t;
        if constexpr (NPL > 0) {
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            const int i = lane + 32 * u;
            if (i < r) {
              ap[i] = cs * xa[u] - sn * ya[u];
              aq[i] = sn * xa[u] + cs * ya[u];
            }
            if (i < c) {
              wp[i] = cs * xw[u] - sn * yw[u];
              wq[i] = sn * xw[u] + cs * yw[u];
            }
          }
        } else {
          for (int i = lane; i < r; i += 32) {
            const float x = ap[i], y = aq[i];
            ap[i] = cs * x - sn * y;
            aq[i] = sn * x + cs * y;
          }
          for (int i = lane; i < c; i += 32) {
            const float x = wp[i], y = wq[i];
            wp[i] = cs * x - sn * y;
            wq[i] = sn * x + cs * y;
          }
        }
        if (lane == 0) rotated_s = 1;
      }
      cl.sync();
    }
    int any = 0;
    for (int qr = 0; qr < SVD_CL; ++qr) any |= *cl.map_shared_rank(&rotated_s, qr);
    cl.sync();
    if (!any) break;
  }
  // Newton-Schulz 1: T1 = W32^T W32 (exact float products, df64 sums); W = W32 (1.5 I - 0.5 T1)
  for (int e = gtid; e < c * c; e += gthreads) {
    const int i = e % c, j = e / c;
    const float* wi = colW(i);
    const float* wj = colW(j);
    df64 a = df_zero();
    for (int q = 0; q < c; ++q) a = df_add(a, two_prod(wi[q], wj[q]));
    T1[(int64_t)j * c + i] = a;
  }
  cl.sync();
  for (int e = gtid; e < c * c; e += gthreads) {
    const int row = e % c, j = e / c;
    df64 a = df_zero();
    for (int i = 0; i < c; ++i) a = df_fma(make_df(colW(i)[row], 0.f), T1[(int64_t)j * c + i], a);
    const df64 wkj = make_df(colW(j)[row], 0.f);
    W[(int64_t)j * c + row] = df_sub(df_mul_f(wkj, 1.5f), df_scale(a, 0.5f));
  }
  cl.sync();
  // Newton-Schulz 2 in df64: T1 = W^T W; A (scratch) = W (1.5 I - 0.5 T1); W = A
  for (int e = gtid; e < c * c; e += gthreads) {
    const int i = e % c, j = e / c;
    const df64* wi = W + (int64_t)i * c;
    const df64* wj = W + (int64_t)j * c;
    df64 a = df_zero();
    for (int q = 0; q < c; ++q) a = df_fma(wi[q], wj[q], a);
    T1[(int64_t)j * c + i] = a;
  }
  cl.sync();
  for (int e = gtid; e < c * c; e += gthreads) {
    const int row = e % c, j = e / c;
    df64 a = df_zero();
    for (int i = 0; i < c; ++i) a = df_fma(W[(int64_t)i * c + row], T1[(int64_t)j * c + i], a);
    A[(int64_t)j * c + row] = df_sub(df_mul_f(W[(int64_t)j * c + row], 1.5f), df_scale(a, 0.5f));
  }
  cl.sync();
  for (int e = gtid; e < c * c; e += gthreads) W[e] = A[e];
  cl.sync();
  // A = B[:r, :c] W
  for (int e = gtid; e < r * c; e += gthreads) {
    const int i = e % r, j = e / r;
    df64 a = df_zero();
    for (int q = 0; q < c; ++q) a = df_fma(B[(int64_t)i * ldb + q], W[(int64_t)j * c + q], a);
    A[(int64_t)j * r + i] = a;
  }
}

__global__ void __launch_bounds__(PRE_THREADS) k_svd_precondition(const df64* __restrict__ B, int ldb, int r, int c,
                                                                  df64* __restrict__ A, df64* __restrict__ W,
                                                                  df64* __restrict__ T1, int cc, int max_sweeps,
                                                                  float tol32) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* A32 = reinterpret_cast<float*>(smem_raw);
  float* W32 = A32 + (size_t)r * c;
  svd_precondition_body<PRE_THREADS>(B, ldb, r, c, A, W, T1, cc, max_sweeps, tol32, A32, W32);
}

// Thick restart: B <- [diag(sigma_1..sigma_kk) | rho], rho_i = alpha_res P[r-1, i].
__global__ void k_restart_B(df64* B, int ldb, int nrows_clear, const df64* __restrict__ sigma,
                            const df64* __restrict__ P, int r, int kk, df64 alpha_res_unused, int c_old) {
  // alpha_res sits at B[r-1][c_old]; read it before clearing
  __shared__ df64 ar;
  if (threadIdx.x == 0) ar = B[(int64_t)(r - 1) * ldb + c_old];
  __syncthreads();
  for (int e = threadIdx.x; e < nrows_clear * ldb; e += blockDim.x) B[e] = df_zero();
  __syncthreads();
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {
    B[(int64_t)i * ldb + i] = sigma[i];
    B[(int64_t)i * ldb + kk] = df_mul(ar, P[(int64_t)i * r + (r - 1)]);
  }
  (void)alpha_res_unused;
}

// out[:, m] = sum_{i<r} Q[:, i] P[i, m] for m < ncol (P col-major with leading dim ldp).
// A block owns RZ_COLS output columns (blockIdx.x, fastest, so the column
// groups of the same rows run together and share the rows of Q in L2) and
// walks row blocks of 512 (blockIdx.y, grid-stride); each thread keeps a
// 2-row x RZ_COLS register tile of lazy double-float accumulators,
// renormalised every 32 terms, and loads its next row pair of Q one
// iteration ahead; P's slice sits in shared memory as [i][m].
constexpr int RZ_COLS = 16;
__global__ void __launch_bounds__(256) k_ritz(const df64* __restrict__ Q, int64_t ldq, int r,
                                              const df64* __restrict__ P, int ldp, int ncol,
                                              df64* __restrict__ out, int64_t ldo, int64_t dim) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df64* Ps = reinterpret_cast<df64*>(smem_raw);  // [r][RZ_COLS]
  const int m0 = blockIdx.x * RZ_COLS;
  for (int e = threadIdx.x; e < r * RZ_COLS; e += blockDim.x) {
    const int i = e / RZ_COLS, mm = e % RZ_COLS;
    Ps[e] = (m0 + mm < ncol) ? P[(int64_t)(m0 + mm) * ldp + i] : df_zero();
  }
  __syncthreads();
  const int64_t nrb = (dim + 511) / 512;
  for (int64_t rb = blockIdx.y; rb < nrb; rb += gridDim.y) {
    const int64_t row = rb * 512 + 2 * threadIdx.x;
    dacc acc[2][RZ_COLS];
#pragma unroll
    for (int m = 0; m < RZ_COLS; ++m) acc[0][m] = acc[1][m] = dacc_zero();
    if (row < dim) {
      const df64* qr = Q + row;
      float4 qn = ld_pair(qr, 0, dim - row);  // the next row pair, one iteration ahead
      for (int i = 0; i < r; ++i) {
        const float4 q = qn;
        if (i + 1 < r) qn = ld_pair(qr + (int64_t)(i + 1) * ldq, 0, dim - row);
        const df64 q0 = make_df(q.x, q.y), q1 = make_df(q.z, q.w);
        const float4* pp = reinterpret_cast<const float4*>(Ps + i * RZ_COLS);
#pragma unroll
        for (int mm = 0; mm < RZ_COLS / 2; ++mm) {
          const float4 pv = pp[mm];
          const df64 p0 = make_df(pv.x, pv.y), p1 = make_df(pv.z, pv.w);
          dacc_fma(acc[0][2 * mm], q0, p0);
          dacc_fma(acc[1][2 * mm], q1, p0);
          dacc_fma(acc[0][2 * mm + 1], q0, p1);
          dacc_fma(acc[1][2 * mm + 1], q1, p1);
        }
        if ((i & 31) == 31) {
#pragma unroll
          for (int m = 0; m < RZ_COLS; ++m) {
            dacc_norm(acc[0][m]);
            dacc_norm(acc[1][m]);
          }
        }
      }
#pragma unroll
      for (int m = 0; m < RZ_COLS; ++m) {
        if (m0 + m < ncol) {
          const df64 v0 = dacc_val(acc[0][m]), v1 = dacc_val(acc[1][m]);
          df64* o = out + (int64_t)(m0 + m) * ldo + row;
          if (row + 1 < dim) {
            *reinterpret_cast<float4*>(o) = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
          } else {
            o[0] = v0;
          }
        }
      }
    }
  }
}

__global__ void k_copy_df(const df64* __restrict__ src, df64* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Sign rule: for each column j of U (dim x k), +1 if its entry of largest
// magnitude (lowest index among equals) is positive, else -1.
__global__ void k_sign(const df64* __restrict__ U, int64_t ldu, int64_t dim, int* __restrict__ sgn) {
  const int j = blockIdx.x;
  const df64* u = U + (int64_t)j * ldu;
  df64 best = make_df(-1.f, 0.f);
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) {
    const df64 a = df_abs(u[i]);
    if (df_gt(a, best)) { best = a; bi = i; }
  }
  __shared__ df64 sb[1024];
  __shared__ int64_t si[1024];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if ((int)threadIdx.x < s) {
      const df64 o = sb[threadIdx.x + s];
      const int64_t oi = si[threadIdx.x + s];
      const df64 me = sb[threadIdx.x];
      if (df_gt(o, me) || (o.hi == me.hi && o.lo == me.lo && oi < si[threadIdx.x])) {
        sb[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sgn[j] = u[si[0]].hi < 0.f ? -1 : 1;
}

// Q[:, j] /= ||Q[:, j]|| in place, one block per column (Ritz vectors of a basis
// that is not orthonormal)
__global__ void __launch_bounds__(256) k_normalize_cols(df64* __restrict__ Q, int64_t ldq, int64_t dim) {
  __shared__ df64 sh[32];
  __shared__ df64 s_inv;
  df64* q = Q + (int64_t)blockIdx.x * ldq;
  df64 acc = df_zero();
  for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) acc = df_fma(q[i], q[i], acc);
  acc = block_sum_df(acc, sh);
  if (threadIdx.x == 0) {
    const df64 nrm = df_sqrt(acc);
    s_inv = nrm.hi > 0.f ? df_div(make_df(1.f, 0.f), nrm) : make_df(1.f, 0.f);
  }
  __syncthreads();
  const df64 inv = s_inv;
  for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) q[i] = df_mul(q[i], inv);
}

// dst[:, j] = sgn[j] * src[:, j] as doubles
__global__ void k_store_cols(const df64* __restrict__ src, int64_t lds, int64_t dim, int ncol,
                             const int* __restrict__ sgn, double* __restrict__ dst, int64_t ldd) {
  const int64_t total = dim * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / dim, i = e - j * dim;
    const double v = df_to_double(src[j * lds + i]);
    dst[j * ldd + i] = sgn ? v * sgn[j] : v;
  }
}

__global__ void k_df_to_double(const df64* __restrict__ src, double* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = df_to_double(src[i]);
}
__global__ void k_double_to_df(const double* __restrict__ src, int64_t lds, df64* __restrict__ dst, int64_t ldd,
                               int64_t dim, int ncol) {
  const int64_t total = dim * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / dim, i = e - j * dim;
    dst[j * ldd + i] = df_from_double(src[j * lds + i]);
  }
}

// FP64 column dot products: one block per column, fixed reduction order.
__global__ void __launch_bounds__(256) k_col_dots(const double* __restrict__ A, int64_t lda,
                                                  const double* __restrict__ B, int64_t ldb, int64_t dim,
                                                  double* __restrict__ out) {
  __shared__ double red[8];
  const double* a = A + (int64_t)blockIdx.x * lda;
  const double* b = B + (int64_t)blockIdx.x * ldb;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < dim; i += 256) acc = fma(a[i], b[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- launchers
static int grid_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

int coop_blocks() {
  static const int blocks = [] {  // thread-safe one-time initialisation
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_normalize_coop, 256, 0);
    if (per < 1) per = 1;
    if (per > 4) per = 4;
    return sms * per;
  }();
  return blocks;
}

int launch_normalize_coop(df64* w, int64_t dim, ReorthWork& rw, df64* qcol, df64* bentry, df64* est,
                          const df64* Q, int64_t ldq, int ncols, uint64_t seed, uint64_t stream, unsigned* status,
                          cudaStream_t s) {
  int blocks = grid_for(dim, 256, coop_blocks());
  if (rw.grid_cap > 0 && blocks > rw.grid_cap) blocks = rw.grid_cap;
  int lds = MAXCOL + 1;
  const df64* nrm = rw.nrm;
  df64* scratch = rw.coop;
  const df64* npart = rw.part2;
  int nblk = rw.nrm_blocks, ldnp = rw.ldp2, ncol = rw.nrm_col;
  const int* ngate = rw.nrm_gate;
  const int* skipf = ncols > 0 ? rw.skip_flag : nullptr;
  const df64* hproj = rw.h;
  void* args[] = {&w,    &dim,  &nrm,    &qcol,   &bentry, &est,  &Q,    &ldq,  &ncols, &scratch, &lds,
                  &seed, &stream, &status, &npart,  &nblk, &ldnp, &ncol, &ngate, &skipf, &hproj};
  prof_begin(s);
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_normalize_coop, dim3(blocks), dim3(256), args, 0, s);
  prof_end(s, K_NORMALIZE, 16.0 * dim, 0.0);
  return e == cudaSuccess ? 0 : (int)e;
}

int launch_pro_pre(df64* w, int64_t dim, const df64* qprev, const df64* coef, ReorthWork& rw, ProState& ps,
                   const df64* B, int ldb, int side, int newidx, int src, int cnt_same, int cnt_other, int prev,
                   const df64* est, cudaStream_t s) {
  ProArgs a{};
  a.w = w;
  a.dim = dim;
  a.qprev = qprev;
  a.coef = coef;
  a.nrm = rw.nrm;
  a.run = rw.run;
  a.gate = rw.gate;
  a.M = ps.M;
  a.N = ps.N;
  a.lde = ps.lde;
  a.B = B;
  a.ldb = ldb;
  a.side = side;
  a.newidx = newidx;
  a.src = src;
  a.cnt_same = cnt_same;
  a.cnt_other = cnt_other;
  a.prev = prev;
  a.eps = ps.eps;
  a.est = est;
  a.force = ps.force;
  a.scratch = rw.coop;
  a.lds = MAXCOL + 1;
  static const int pro_cap = [] {  // co-resident blocks of this kernel (its own occupancy)
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pro_pre, 256, 0);
    if (per < 1) per = 1;
    return sms * per < coop_blocks() ? sms * per : coop_blocks();
  }();
  int blocks = grid_for(dim, 256, pro_cap);
  if (rw.grid_cap > 0 && blocks > rw.grid_cap) blocks = rw.grid_cap;
  void* args[] = {&a};
  prof_begin(s);
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_pro_pre, dim3(blocks), dim3(256), args, 0, s);
  prof_end(s, K_MISC, qprev ? 24.0 * dim : 16.0 * dim, 0.0);
  return e == cudaSuccess ? 0 : (int)e;
}

void launch_pro_reset(ProState& ps, cudaStream_t s) {
  k_pro_reset<<<64, 256, 0, s>>>(ps.M, ps.N, ps.lde, ps.lde, ps.eps, ps.force);
}

void launch_random_fill(df64* w, int64_t dim, uint64_t seed, uint64_t stream, cudaStream_t s) {
  prof_begin(s);
  k_random_fill<<<grid_for(dim, 256, 1184), 256, 0, s>>>(w, dim, seed, stream);
  prof_end(s, K_MISC, 8.0 * dim, 0.0);
}

// shared-memory limits of the cluster kernels, once per process
static std::once_flag g_svd_cluster_once;
static void svd_cluster_setup() {
  std::call_once(g_svd_cluster_once, [] {
    cudaFuncSetAttribute(k_svd_precondition_cluster<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, PRE_SMEM_MAX);
    cudaFuncSetAttribute(k_svd_precondition_cluster<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, PRE_SMEM_MAX);
    cudaFuncSetAttribute(k_svd_precondition_cluster<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, PRE_SMEM_MAX);
    cudaFuncSetAttribute(k_small_svd_cluster<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SVD_STAGE_MAX);
    cudaFuncSetAttribute(k_small_svd_cluster<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, SVD_STAGE_MAX);
    cudaFuncSetAttribute(k_small_svd_cluster<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, SVD_STAGE_MAX);
  });
}

void launch_small_svd(const df64* B, int ldb, int r, int c, SvdWork& sw, int k, double tol_conv,
                      df64* est, unsigned* status, cudaStream_t s) {
  const int cc = c + (c & 1);
  const size_t pre_sm = ((size_t)r * c + (size_t)c * c) * sizeof(float);
  int warm = 0;
  const int nloc_p = (c + SVD_CL - 1) / SVD_CL;
  const size_t pre_cl_sm = (size_t)nloc_p * (r + c) * sizeof(float);
  // column pieces per lane held in registers by the cluster kernels (0: loops over shared memory)
  const int npl = ((r > c ? r : c) + 31) / 32;
  svd_cluster_setup();
  if (c >= 16 && pre_cl_sm <= (size_t)PRE_SMEM_MAX) {
    prof_begin(s);
    if (npl <= 4)
      k_svd_precondition_cluster<4><<<SVD_CL, SVD_CL_THREADS, pre_cl_sm, s>>>(B, ldb, r, c, sw.A, sw.W, sw.P, cc,
                                                                              PRE_SWEEPS, 2e-6f);
    else if (npl <= 8)
      k_svd_precondition_cluster<8><<<SVD_CL, SVD_CL_THREADS, pre_cl_sm, s>>>(B, ldb, r, c, sw.A, sw.W, sw.P, cc,
                                                                              PRE_SWEEPS, 2e-6f);
    else
      k_svd_precondition_cluster<0><<<SVD_CL, SVD_CL_THREADS, pre_cl_sm, s>>>(B, ldb, r, c, sw.A, sw.W, sw.P, cc,
                                                                              PRE_SWEEPS, 2e-6f);
    prof_end(s, K_SVD_PRE, 0.0, 0.0);
    warm = 1;
  } else if (c >= 16 && pre_sm <= (size_t)PRE_SMEM_MAX) {
    static std::once_flag attr;
    std::call_once(attr, [] {
      cudaFuncSetAttribute(k_svd_precondition, cudaFuncAttributeMaxDynamicSharedMemorySize, PRE_SMEM_MAX);
    });
    prof_begin(s);
    // FP32 sweeps stop improving near FP32 resolution; the df64 sweeps finish from there
    k_svd_precondition<<<1, PRE_THREADS, pre_sm, s>>>(B, ldb, r, c, sw.A, sw.W, sw.P, cc, PRE_SWEEPS, 2e-6f);
    prof_end(s, K_SVD_PRE, 0.0, 0.0);
    warm = 1;
  }
  // the cluster version when its share of the columns fits in each CTA
  const int nloc = (c + SVD_CL - 1) / SVD_CL;
  const size_t cl_sm = ((size_t)nloc * (r + c) + nloc) * sizeof(df64);
  if (cl_sm <= (size_t)SVD_STAGE_MAX) {
    prof_begin(s);
#define SSA_SVD_CL(NPL)                                                                                        \
  k_small_svd_cluster<NPL><<<SVD_CL, SVD_CL_THREADS, cl_sm, s>>>(B, ldb, r, c, sw.A, sw.W, cc, sw.sigma, sw.P,  \
                                                                 sw.Q, sw.resid, sw.sigma_d, k, tol_conv, sw.conv, \
                                                                 est, status, sw.max_sweeps, sw.rot_tol, warm)
    if (npl <= 4) SSA_SVD_CL(4);
    else if (npl <= 8) SSA_SVD_CL(8);
    else SSA_SVD_CL(0);
#undef SSA_SVD_CL
    prof_end(s, K_SMALL_SVD, 0.0, 0.0);
    return;
  }
  const size_t st_sm = ((size_t)r * c + (size_t)c * c) * sizeof(df64);
  const int staged = st_sm <= (size_t)SVD_STAGE_MAX ? 1 : 0;
  static std::once_flag attr2;
  std::call_once(attr2, [] {
    cudaFuncSetAttribute(k_small_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, SVD_STAGE_MAX);
  });
  prof_begin(s);
  k_small_svd<<<1, SVD_THREADS, staged ? st_sm : 0, s>>>(B, ldb, r, c, sw.A, sw.W, cc, sw.sigma, sw.P, sw.Q,
                                                         sw.resid, sw.sigma_d, k, tol_conv, sw.conv, est, status,
                                                         sw.max_sweeps, sw.rot_tol, warm, staged);
  prof_end(s, K_SMALL_SVD, 0.0, 0.0);
}

void launch_restart_B(df64* B, int ldb, int nrows_clear, const SvdWork& sw, int r, int kk, int c_old,
                      cudaStream_t s) {
  prof_begin(s);
  k_restart_B<<<1, 512, 0, s>>>(B, ldb, nrows_clear, sw.sigma, sw.P, r, kk, df_zero(), c_old);
  prof_end(s, K_MISC, 0.0, 0.0);
}

void launch_ritz(const df64* Q, int64_t ldq, int r, const df64* P, int ldp, int ncol, df64* out, int64_t ldo,
                 int64_t dim, cudaStream_t s) {
  const int64_t nrb = (dim + 511) / 512;
  dim3 grid((unsigned)((ncol + RZ_COLS - 1) / RZ_COLS), (unsigned)(nrb < 65535 ? nrb : 65535));
  const size_t sm = (size_t)r * RZ_COLS * sizeof(df64);
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(MAXCOL + 2) * RZ_COLS * 8);
  });
  prof_begin(s);
  k_ritz<<<grid, 256, sm, s>>>(Q, ldq, r, P, ldp, ncol, out, ldo, dim);
  prof_end(s, K_RITZ, 8.0 * (double)dim * (r + ncol), 2.0 * (double)dim * r * ncol);
}

void launch_copy_df(const df64* src, df64* dst, int64_t n, cudaStream_t s) {
  prof_begin(s);
  k_copy_df<<<grid_for(n, 256, 1184), 256, 0, s>>>(src, dst, n);
  prof_end(s, K_MISC, 16.0 * n, 0.0);
}

void launch_sign(const df64* U, int64_t ldu, int64_t dim, int k, int* sgn, cudaStream_t s) {
  prof_begin(s);
  k_sign<<<k, 1024, 0, s>>>(U, ldu, dim, sgn);
  prof_end(s, K_MISC, 8.0 * (double)dim * k, 0.0);
}

void launch_normalize_cols(df64* Q, int64_t ldq, int64_t dim, int ncol, cudaStream_t s) {
  if (ncol <= 0) return;
  prof_begin(s);
  k_normalize_cols<<<ncol, 256, 0, s>>>(Q, ldq, dim);
  prof_end(s, K_MISC, 16.0 * (double)dim * ncol, 0.0);
}

void launch_store_cols(const df64* src, int64_t lds, int64_t dim, int ncol, const int* sgn, double* dst, int64_t ldd,
                       cudaStream_t s) {
  prof_begin(s);
  k_store_cols<<<grid_for(dim * ncol, 256, 4736), 256, 0, s>>>(src, lds, dim, ncol, sgn, dst, ldd);
  prof_end(s, K_MISC, 16.0 * (double)dim * ncol, 0.0);
}

void launch_col_dots(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t dim, int ncol, double* out,
                     cudaStream_t s) {
  prof_begin(s);
  k_col_dots<<<ncol, 256, 0, s>>>(A, lda, B, ldb, dim, out);
  prof_end(s, K_MISC, 16.0 * (double)dim * ncol, 2.0 * (double)dim * ncol);
}

void launch_df_to_double(const df64* src, double* dst, int64_t n, cudaStream_t s) {
  prof_begin(s);
  k_df_to_double<<<grid_for(n, 256, 1184), 256, 0, s>>>(src, dst, n);
  prof_end(s, K_MISC, 16.0 * n, 0.0);
}

void launch_double_to_df(const double* src, int64_t lds, df64* dst, int64_t ldd, int64_t dim, int ncol,
                         cudaStream_t s) {
  prof_begin(s);
  k_double_to_df<<<grid_for(dim * ncol, 256, 4736), 256, 0, s>>>(src, lds, dst, ldd, dim, ncol);
  prof_end(s, K_MISC, 16.0 * (double)dim * ncol, 0.0);
}

}  // namespace ssa
