// Device kernels of the Golub-Kahan-Lanczos engine (section 3): full
// reorthogonalisation by classical Gram-Schmidt applied twice (CGS2), the
// normalisation with breakdown replacement, the SVD of the projected matrix B
// by one-sided Jacobi in one CTA, the Ritz-vector products U P and V Q of a
// thick restart, and the output conversion with the sign rule.  All vectors
// and the projected problem are double-float (df64).
#include <cooperative_groups.h>
#include "lanczos.h"
#include "prof.h"

namespace ssa {

SSA_D df64 shfl_xor_df(df64 v, int m) {
  return make_df(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
// df_add is commutative bit-for-bit, so the butterfly leaves the same sum in every lane.
SSA_D df64 warp_sum_df(df64 v) {
#pragma unroll
  for (int m = 16; m; m >>= 1) v = df_add(v, shfl_xor_df(v, m));
  return v;
}

SSA_D float4 ld_pair(const df64* p, int64_t row, int64_t dim) {
  // two consecutive rows (row even, 16-byte aligned); rows >= dim read as 0
  if (row + 1 < dim) return __ldg(reinterpret_cast<const float4*>(p + row));
  if (row < dim) {
    df64 a = p[row];
    return make_float4(a.hi, a.lo, 0.f, 0.f);
  }
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

// Block-level end of a two-stage reduction: every block writes its partials,
// the last block to finish sums them in block order (deterministic) and
// resets the counter.
SSA_D bool last_block(int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  return is_last;
}

// ---------------------------------------------------------------- CGS pieces
// h[i] = Q[:, i] . w for i < ncols and h[ncols] = w . w
__global__ void __launch_bounds__(RT) k_proj(const df64* __restrict__ Q, int64_t ldq, int ncols,
                                             const df64* __restrict__ w, int64_t dim, df64* __restrict__ part,
                                             int ldp, df64* __restrict__ hout, int* counter, const int* flag) {
  if (flag && *flag == 0) return;
  __shared__ df64 red[RT / 32][MAXCOL + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * SLAB;
  df64 wv[RP][2];
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
    float4 v = ld_pair(w, row, dim);
    wv[p][0] = make_df(v.x, v.y);
    wv[p][1] = make_df(v.z, v.w);
  }
  for (int i = 0; i <= ncols; ++i) {
    df64 acc = df_zero();
    if (i < ncols) {
      const df64* q = Q + (int64_t)i * ldq;
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
        float4 v = ld_pair(q, row, dim);
        acc = df_fma(make_df(v.x, v.y), wv[p][0], acc);
        acc = df_fma(make_df(v.z, v.w), wv[p][1], acc);
      }
    } else {
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        acc = df_fma(wv[p][0], wv[p][0], acc);
        acc = df_fma(wv[p][1], wv[p][1], acc);
      }
    }
    acc = warp_sum_df(acc);
    if (lane == 0) red[warp][i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= ncols; i += RT) {
    df64 s = df_zero();
#pragma unroll
    for (int wp = 0; wp < RT / 32; ++wp) s = df_add(s, red[wp][i]);
    part[(int64_t)blockIdx.x * ldp + i] = s;
  }
  if (last_block(counter)) {
    for (int i = threadIdx.x; i <= ncols; i += RT) {
      df64 s = df_zero();
      for (int b = 0; b < (int)gridDim.x; ++b) {
        const volatile df64* pp = part + (int64_t)b * ldp + i;
        s = df_add(s, make_df(pp->hi, pp->lo));
      }
      hout[i] = s;
    }
    if (threadIdx.x == 0) *counter = 0;
  }
}

// w -= Q[:, :ncols] h ; nrm_out = w . w
__global__ void __launch_bounds__(RT) k_update(const df64* __restrict__ Q, int64_t ldq, int ncols,
                                               df64* __restrict__ w, int64_t dim, const df64* __restrict__ h,
                                               df64* __restrict__ part, df64* __restrict__ nrm_out, int* counter,
                                               const int* flag) {
  if (flag && *flag == 0) return;
  __shared__ df64 hs[MAXCOL + 1];
  __shared__ df64 red[RT / 32];
  for (int i = threadIdx.x; i < ncols; i += RT) hs[i] = h[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * SLAB;
  df64 acc[RP][2];
#pragma unroll
  for (int p = 0; p < RP; ++p) acc[p][0] = acc[p][1] = df_zero();
  for (int i = 0; i < ncols; ++i) {
    const df64 hi = hs[i];
    const df64* q = Q + (int64_t)i * ldq;
#pragma unroll
    for (int p = 0; p < RP; ++p) {
      const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
      float4 v = ld_pair(q, row, dim);
      acc[p][0] = df_fma(make_df(v.x, v.y), hi, acc[p][0]);
      acc[p][1] = df_fma(make_df(v.z, v.w), hi, acc[p][1]);
    }
  }
  df64 nrm = df_zero();
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (row + e < dim) {
        df64 x = df_sub(w[row + e], acc[p][e]);
        w[row + e] = x;
        nrm = df_fma(x, x, nrm);
      }
    }
  }
  nrm = warp_sum_df(nrm);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    df64 s = df_zero();
    for (int wp = 0; wp < RT / 32; ++wp) s = df_add(s, red[wp]);
    part[blockIdx.x] = s;
  }
  if (last_block(counter)) {
    if (threadIdx.x == 0) {
      df64 s = df_zero();
      for (int b = 0; b < (int)gridDim.x; ++b) {
        const volatile df64* pp = part + b;
        s = df_add(s, make_df(pp->hi, pp->lo));
      }
      *nrm_out = s;
      *counter = 0;
    }
  }
}

// ---------------------------------------------------------------- random vectors
SSA_D uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// uniform in [-1, 1) from splitmix64 in counter mode (stream s, index i)
SSA_D df64 sm64_uniform_pm1(uint64_t seed, uint64_t stream, int64_t i) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  const uint64_t key = sm64_mix(seed + (stream + 1) * G);
  const uint64_t z = sm64_mix(key + ((uint64_t)i + 1) * G);
  // 53-bit uniform u; 2u - 1 split into two floats exactly enough for df64
  const int64_t m = (int64_t)(z >> 11) - ((int64_t)1 << 52);  // 2u-1 = m * 2^-52
  const float hi = (float)(m >> 29) * 0x1p-23f;
  const float lo = (float)(m & ((1 << 29) - 1)) * 0x1p-52f;
  return fast_two_sum(hi, lo);
}

__global__ void k_random_fill(df64* w, int64_t dim, uint64_t seed, uint64_t stream) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = sm64_uniform_pm1(seed, stream, i);
}

// Normalise w into column qcol and record the coupling coefficient.
//   mode 0: beta = sqrt(nrm2); if beta <= 1e-14 * est (breakdown, including
//           beta == 0) the coefficient is recorded as 0, w is replaced by a
//           seeded random vector and *flag = 1 so that the conditional
//           reorthogonalisation that follows runs; otherwise *flag = 0.
//   mode 1: only when *flag: normalise the reorthogonalised random vector;
//           if it vanished (the basis already spans the space) store zeros.
// est (largest coupling / singular value seen) is raised by block 0 at the
// end; other blocks may read the old or the new value, which gives the same
// decision because the new value is beta itself.
__global__ void k_normalize(df64* __restrict__ w, int64_t dim, const df64* __restrict__ nrm2,
                            df64* __restrict__ qcol, df64* __restrict__ bentry, df64* est, int* flag, int mode,
                            uint64_t seed, uint64_t stream, unsigned* status) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (mode == 1 && *flag == 0) return;
  const df64 beta = df_sqrt(*nrm2);
  if (!isfinite(beta.hi)) {
    if (tid == 0) atomicOr(status, SSA_DEV_NONFINITE);
  }
  if (mode == 0) {
    const float thr = 1e-14f * est->hi;
    if (beta.hi > thr && beta.hi > 0.f && isfinite(beta.hi)) {
      const df64 inv = df_div(make_df(1.f, 0.f), beta);
      for (int64_t i = tid; i < dim; i += stride) qcol[i] = df_mul(w[i], inv);
      __syncthreads();
      if (tid == 0) {
        *bentry = beta;
        if (df_gt(beta, *est)) *est = beta;
        *flag = 0;
      }
    } else {
      for (int64_t i = tid; i < dim; i += stride) w[i] = sm64_uniform_pm1(seed, stream, i);
      if (tid == 0) {
        *bentry = df_zero();
        *flag = 1;
        atomicOr(status, SSA_DEV_BREAKDOWN);
      }
    }
  } else {
    // the random vector had norm ~ sqrt(dim/3) before orthogonalisation
    const float ref = sqrtf((float)dim / 3.f);
    const bool alive = beta.hi > 1e-6f * ref;
    const df64 inv = alive ? df_div(make_df(1.f, 0.f), beta) : df_zero();
    for (int64_t i = tid; i < dim; i += stride) qcol[i] = df_mul(w[i], inv);
  }
}

__global__ void k_clear_flag(int* flag) { *flag = 0; }

// ---------------------------------------------------------------- projected SVD
// One-sided Jacobi (Hestenes) on the r x c block of B (row-major, leading
// dimension ldb), in one CTA.  Parallel ordering: the host supplies a
// round-robin schedule (cc-1 rounds of cc/2 disjoint pairs, cc = c rounded up
// to even; index c is a dummy).  Each warp rotates one pair at a time.
// Outputs (col-major): P (r x c) left singular vectors, Qv (c x c) right,
// sigma (c), all sorted by descending sigma; resid[m] = |alpha_res P[r-1, m]|;
// *conv = all(resid[m] <= tol_conv * sigma[0], m < k).
__global__ void __launch_bounds__(SVD_THREADS) k_small_svd(const df64* __restrict__ B, int ldb, int r, int c,
                                                           df64* __restrict__ A, df64* __restrict__ W,
                                                           const int2* __restrict__ sched, int cc,
                                                           df64* __restrict__ sigma, df64* __restrict__ P,
                                                           df64* __restrict__ Qv, double* __restrict__ resid,
                                                           double* __restrict__ sigma_d, int k, double tol_conv,
                                                           int* conv, df64* est, unsigned* status, int max_sweeps,
                                                           float rot_tol) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = SVD_THREADS / 32;
  __shared__ int rotated;
  __shared__ int sweeps_used;
  // A = B[:r, :c] in column-major, W = I
  for (int e = threadIdx.x; e < r * c; e += SVD_THREADS) {
    const int i = e % r, j = e / r;
    A[(int64_t)j * r + i] = B[(int64_t)i * ldb + j];
  }
  for (int e = threadIdx.x; e < c * c; e += SVD_THREADS) {
    const int i = e % c, j = e / c;
    W[(int64_t)j * c + i] = make_df(i == j ? 1.f : 0.f, 0.f);
  }
  if (threadIdx.x == 0) sweeps_used = -1;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < cc - 1; ++rnd) {
      for (int pr = warp; pr < cc / 2; pr += nw) {
        const int2 pq = sched[(int64_t)rnd * (cc / 2) + pr];
        const int p = pq.x, q = pq.y;
        if (p >= c || q >= c) continue;
        df64* ap = A + (int64_t)p * r;
        df64* aq = A + (int64_t)q * r;
        df64 al = df_zero(), be = df_zero(), ga = df_zero();
        for (int i = lane; i < r; i += 32) {
          const df64 x = ap[i], y = aq[i];
          al = df_fma(x, x, al);
          be = df_fma(y, y, be);
          ga = df_fma(x, y, ga);
        }
        al = warp_sum_df(al);
        be = warp_sum_df(be);
        ga = warp_sum_df(ga);
        if (!(al.hi > 0.f) || !(be.hi > 0.f)) continue;
        // rotate when |gamma| > tol sqrt(alpha) sqrt(beta) (square roots keep
        // the test inside the float exponent range)
        const df64 thr = df_mul_f(df_mul(df_sqrt(al), df_sqrt(be)), rot_tol);
        if (!df_gt(df_abs(ga), thr)) continue;
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
        for (int i = lane; i < r; i += 32) {
          const df64 x = ap[i], y = aq[i];
          ap[i] = df_sub(df_mul(cs, x), df_mul(sn, y));
          aq[i] = df_add(df_mul(sn, x), df_mul(cs, y));
        }
        df64* wp = W + (int64_t)p * c;
        df64* wq = W + (int64_t)q * c;
        for (int i = lane; i < c; i += 32) {
          const df64 x = wp[i], y = wq[i];
          wp[i] = df_sub(df_mul(cs, x), df_mul(sn, y));
          wq[i] = df_add(df_mul(sn, x), df_mul(cs, y));
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) {
      if (threadIdx.x == 0) sweeps_used = sweep + 1;
      break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && sweeps_used < 0) atomicOr(status, SSA_DEV_JACOBI_NOCONV);
  // column norms -> sigma (stored temporarily in sigma[] unsorted)
  for (int j = warp; j < c; j += nw) {
    df64 s = df_zero();
    for (int i = lane; i < r; i += 32) s = df_fma(A[(int64_t)j * r + i], A[(int64_t)j * r + i], s);
    s = warp_sum_df(s);
    if (lane == 0) sigma[j] = df_sqrt(s);
  }
  __syncthreads();
  // rank by descending sigma (ties: lower index first) and scatter
  __shared__ int rank_of[MAXCOL + 2];
  for (int j = threadIdx.x; j < c; j += SVD_THREADS) {
    const df64 sj = sigma[j];
    int rk = 0;
    for (int i = 0; i < c; ++i) {
      const df64 si = sigma[i];
      if (df_gt(si, sj) || (si.hi == sj.hi && si.lo == sj.lo && i < j)) ++rk;
    }
    rank_of[j] = rk;
  }
  __syncthreads();
  for (int j = warp; j < c; j += nw) {
    const int rk = rank_of[j];
    const df64 sj = sigma[j];
    const df64 inv = sj.hi > 0.f ? df_div(make_df(1.f, 0.f), sj) : df_zero();
    for (int i = lane; i < r; i += 32) P[(int64_t)rk * r + i] = df_mul(A[(int64_t)j * r + i], inv);
    for (int i = lane; i < c; i += 32) Qv[(int64_t)rk * c + i] = W[(int64_t)j * c + i];
  }
  __syncthreads();
  // sorted sigma: reuse A's first column as scratch is unsafe; write via rank
  __shared__ df64 ssort[MAXCOL + 2];
  for (int j = threadIdx.x; j < c; j += SVD_THREADS) ssort[rank_of[j]] = sigma[j];
  __syncthreads();
  for (int j = threadIdx.x; j < c; j += SVD_THREADS) {
    sigma[j] = ssort[j];
    sigma_d[j] = df_to_double(ssort[j]);
  }
  __syncthreads();
  // residuals from relation (2) and the convergence test
  const df64 alpha_res = B[(int64_t)(r - 1) * ldb + c];
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  const double s1 = df_to_double(ssort[0]);
  for (int m = threadIdx.x; m < c; m += SVD_THREADS) {
    const double rm = fabs(df_to_double(df_mul(alpha_res, P[(int64_t)m * r + (r - 1)])));
    resid[m] = rm;
    if (m < k && !(rm <= tol_conv * s1)) ok = 0;
    if (!isfinite(rm)) atomicOr(status, SSA_DEV_NONFINITE);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *conv = ok;
    if (df_gt(ssort[0], *est)) *est = ssort[0];
  }
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

// out[:, m] = sum_{i<r} Q[:, i] P[i, m] for m < ncol (P col-major with leading dim ldp)
__global__ void __launch_bounds__(256) k_ritz(const df64* __restrict__ Q, int64_t ldq, int r,
                                              const df64* __restrict__ P, int ldp, int ncol,
                                              df64* __restrict__ out, int64_t ldo, int64_t dim) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df64* Pt = reinterpret_cast<df64*>(smem_raw);  // [r][32]
  const int m0 = blockIdx.y * 32;
  for (int e = threadIdx.x; e < r * 32; e += blockDim.x) {
    const int i = e >> 5, mm = e & 31;
    Pt[e] = (m0 + mm < ncol) ? P[(int64_t)(m0 + mm) * ldp + i] : df_zero();
  }
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * 64 + (threadIdx.x & 63);
  const int cg = threadIdx.x >> 6;
  df64 acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = df_zero();
  if (row < dim) {
    for (int i = 0; i < r; ++i) {
      const df64 q = Q[(int64_t)i * ldq + row];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = df_fma(q, Pt[i * 32 + cg + 4 * j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int m = m0 + cg + 4 * j;
      if (m < ncol) out[(int64_t)m * ldo + row] = acc[j];
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

// ---------------------------------------------------------------- launchers
static int grid_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

int reorth_blocks(int64_t dim) { return (int)((dim + SLAB - 1) / SLAB); }

// CGS2: w <- (I - Q Q^T)^2 w, nrm2 <- ||w||^2.  flag (may be null) gates the
// whole sequence on the device (used for the breakdown replacement).
void launch_cgs2(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, ReorthWork& rw, const int* flag,
                 cudaStream_t s) {
  const int G = reorth_blocks(dim);
  // algorithmic bytes: the ncols basis columns once, w read (and written by the update)
  const double qb = 8.0 * (double)dim * ncols;
  const double fl = 2.0 * (double)dim * ncols;
  if (ncols > 0) {
    prof_begin(s);
    k_proj<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.part, rw.ldp, rw.h, rw.counter, flag);
    prof_end(s, flag ? K_GATED : K_PROJ, flag ? 0.0 : qb + 8.0 * dim, flag ? 0.0 : fl);
    prof_begin(s);
    k_update<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.h, rw.part, rw.nrm, rw.counter, flag);
    prof_end(s, flag ? K_GATED : K_UPDATE, flag ? 0.0 : qb + 16.0 * dim, flag ? 0.0 : fl);
    prof_begin(s);
    k_proj<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.part, rw.ldp, rw.h, rw.counter, flag);
    prof_end(s, flag ? K_GATED : K_PROJ, flag ? 0.0 : qb + 8.0 * dim, flag ? 0.0 : fl);
  }
  prof_begin(s);
  k_update<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.h, rw.part, rw.nrm, rw.counter, flag);
  prof_end(s, flag ? K_GATED : K_UPDATE, flag ? 0.0 : qb + 16.0 * dim, flag ? 0.0 : fl);
}

void launch_normalize(df64* w, int64_t dim, ReorthWork& rw, df64* qcol, df64* bentry, df64* est, int* flag, int mode,
                      uint64_t seed, uint64_t stream, unsigned* status, cudaStream_t s) {
  prof_begin(s);
  k_normalize<<<grid_for(dim, 256, 1184), 256, 0, s>>>(w, dim, rw.nrm, qcol, bentry, est, flag, mode, seed, stream,
                                                       status);
  prof_end(s, mode == 0 ? K_NORMALIZE : K_GATED, mode == 0 ? 16.0 * dim : 0.0, 0.0);
}

void launch_random_fill(df64* w, int64_t dim, uint64_t seed, uint64_t stream, cudaStream_t s) {
  prof_begin(s);
  k_random_fill<<<grid_for(dim, 256, 1184), 256, 0, s>>>(w, dim, seed, stream);
  prof_end(s, K_MISC, 8.0 * dim, 0.0);
}

void launch_small_svd(const df64* B, int ldb, int r, int c, const int2* sched, SvdWork& sw, int k, double tol_conv,
                      df64* est, unsigned* status, cudaStream_t s) {
  const int cc = c + (c & 1);
  prof_begin(s);
  k_small_svd<<<1, SVD_THREADS, 0, s>>>(B, ldb, r, c, sw.A, sw.W, sched, cc, sw.sigma, sw.P, sw.Q, sw.resid,
                                         sw.sigma_d, k, tol_conv, sw.conv, est, status, sw.max_sweeps, sw.rot_tol);
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
  dim3 grid((unsigned)((dim + 63) / 64), (unsigned)((ncol + 31) / 32));
  const size_t sm = (size_t)r * 32 * sizeof(df64);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(MAXCOL + 2) * 32 * 8);
    attr = true;
  }
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

void launch_store_cols(const df64* src, int64_t lds, int64_t dim, int ncol, const int* sgn, double* dst, int64_t ldd,
                       cudaStream_t s) {
  prof_begin(s);
  k_store_cols<<<grid_for(dim * ncol, 256, 4736), 256, 0, s>>>(src, lds, dim, ncol, sgn, dst, ldd);
  prof_end(s, K_MISC, 16.0 * (double)dim * ncol, 0.0);
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
