// Device building blocks shared by the per-series kernels (lanczos_kernels.cu)
// and the batched persistent kernel (batch.cu): warp/block reductions of
// double-float values, asynchronous copies, the lazy double-float
// accumulator, splitmix64, and the one-CTA projected-SVD bodies.
#pragma once
#include "common.cuh"
#include "lanczos.h"

namespace ssa {

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

// 4-value warp butterfly: on return lane 8*c holds the warp sum of v[c].
SSA_D df64 warp_sum4_df(df64 v0, df64 v1, df64 v2, df64 v3) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8;
  df64 sa = b4 ? v0 : v2, sb = b4 ? v1 : v3;
  df64 ka = b4 ? v2 : v0, kb = b4 ? v3 : v1;
  df64 x0 = df_add(ka, shfl_xor_df(sa, 16));
  df64 x1 = df_add(kb, shfl_xor_df(sb, 16));
  df64 snd = b3 ? x0 : x1, kp = b3 ? x1 : x0;
  df64 u = df_add(kp, shfl_xor_df(snd, 8));
  u = df_add(u, shfl_xor_df(u, 4));
  u = df_add(u, shfl_xor_df(u, 2));
  u = df_add(u, shfl_xor_df(u, 1));
  return u;
}

// Asynchronous 16-byte global->shared copies (LDGSTS); a copy with
// valid == false writes zeros and reads nothing.
SSA_D void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
SSA_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> SSA_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- lazy double-float accumulation: value = hi + lo with lo unnormalised
struct dacc {
  float hi, lo;
};
SSA_D dacc dacc_zero() { return {0.f, 0.f}; }
// s += a * b (12 FP32 instructions; renormalise with dacc_norm every few dozen terms)
SSA_D void dacc_fma(dacc& s, df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + e;
}
SSA_D df64 dacc_val(dacc s) { return fast_two_sum(s.hi, s.lo); }
SSA_D void dacc_norm(dacc& s) {
  const df64 v = fast_two_sum(s.hi, s.lo);
  s.hi = v.hi;
  s.lo = v.lo;
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

// Block sum of one df64 per thread; result valid in thread 0.
SSA_D df64 block_sum_df(df64 v, df64* sh) {
  v = warp_sum_df(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  df64 s = df_zero();
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = df_add(s, sh[i]);
  return s;
}


// Round-robin (circle method) schedule of one-sided Jacobi: cc (even) columns,
// cc-1 rounds of cc/2 disjoint pairs; column 0 stays, the others rotate one
// place per round, so every pair meets once per sweep.
SSA_D int rr_pos(int i, int rnd, int cc) {
  if (i == 0) return 0;
  const int m = cc - 1;
  int v = (i - 1 - rnd) % m;
  if (v < 0) v += m;
  return 1 + v;
}
SSA_D int2 rr_pair(int rnd, int j, int cc) { return make_int2(rr_pos(j, rnd, cc), rr_pos(cc - 1 - j, rnd, cc)); }

// One-sided Jacobi (Hestenes) on the r x c block of B (row-major, leading
// dimension ldb), in one CTA.  Parallel ordering: the host supplies a
// round-robin schedule (cc-1 rounds of cc/2 disjoint pairs, cc = c rounded up
// to even; index c is a dummy).  Each warp rotates one pair at a time.
// Outputs (col-major): P (r x c) left singular vectors, Qv (c x c) right,
// sigma (c), all sorted by descending sigma; resid[m] = |alpha_res P[r-1, m]|;
// *conv = all(resid[m] <= tol_conv * sigma[0], m < k).
template <int THREADS>
SSA_D void svd_jacobi_body(const df64* __restrict__ B, int ldb, int r, int c, df64* __restrict__ A,
                           df64* __restrict__ W, int cc,
                                                           df64* __restrict__ sigma, df64* __restrict__ P,
                                                           df64* __restrict__ Qv, double* __restrict__ resid,
                                                           double* __restrict__ sigma_d, int k, double tol_conv,
                                                           int* conv, df64* est, unsigned* status, int max_sweeps,
                                                           float rot_tol, int warm, df64* stage) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = THREADS / 32;
  __shared__ int rotated;
  __shared__ int sweeps_used;
  __shared__ int ok;
  // With stage (r*c + c*c df64 of shared memory) the sweeps run there: every
  // rotation reads and writes two columns, and L2 latency would dominate.
  if (stage) {
    df64* As = stage;
    df64* Ws = stage + (int64_t)r * c;
    if (warm) {
      for (int e = threadIdx.x; e < r * c; e += THREADS) As[e] = A[e];
      for (int e = threadIdx.x; e < c * c; e += THREADS) Ws[e] = W[e];
    }
    A = As;
    W = Ws;
  }
  // A = B[:r, :c] in column-major, W = I (unless the preconditioner left A = B W, W)
  if (!warm) {
    for (int e = threadIdx.x; e < r * c; e += THREADS) {
      const int i = e % r, j = e / r;
      A[(int64_t)j * r + i] = B[(int64_t)i * ldb + j];
    }
    for (int e = threadIdx.x; e < c * c; e += THREADS) {
      const int i = e % c, j = e / c;
      W[(int64_t)j * c + i] = make_df(i == j ? 1.f : 0.f, 0.f);
    }
  }
  if (threadIdx.x == 0) sweeps_used = -1;
  __syncthreads();
  __shared__ float max_ratio;  // largest |gamma| / sqrt(alpha beta) of the sweep
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      rotated = 0;
      max_ratio = 0.f;
    }
    __syncthreads();
    for (int rnd = 0; rnd < cc - 1; ++rnd) {
      for (int pr = warp; pr < cc / 2; pr += nw) {
        const int2 pq = rr_pair(rnd, pr, cc);
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
        const df64 nab = df_mul(df_sqrt(al), df_sqrt(be));
        const df64 thr = df_mul_f(nab, rot_tol);
        if (!df_gt(df_abs(ga), thr)) continue;
        if (lane == 0) {  // non-negative floats order like their bit patterns
          const float ratio = fabsf(ga.hi) / nab.hi;
          atomicMax(reinterpret_cast<int*>(&max_ratio), __float_as_int(ratio));
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
    const float mr = max_ratio;
    __syncthreads();
    // no rotation, or every rotation of this sweep below 1e-10: with the
    // quadratic convergence of cyclic Jacobi the next sweep's rotations would
    // be far below rot_tol, so that sweep is skipped
    if (!any || mr < 1e-10f) {
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
  for (int j = threadIdx.x; j < c; j += THREADS) {
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
  for (int j = threadIdx.x; j < c; j += THREADS) ssort[rank_of[j]] = sigma[j];
  __syncthreads();
  for (int j = threadIdx.x; j < c; j += THREADS) {
    sigma[j] = ssort[j];
    sigma_d[j] = df_to_double(ssort[j]);
  }
  __syncthreads();
  // residuals from relation (2) and the convergence test
  const df64 alpha_res = B[(int64_t)(r - 1) * ldb + c];
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  const double s1 = df_to_double(ssort[0]);
  for (int m = threadIdx.x; m < c; m += THREADS) {
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


// Preconditioning of the projected SVD (one CTA):
//   1. one-sided Jacobi in FP32 on the rounded r x c block of B, in shared
//      memory, to orthogonality ~1e-6 (cheap sweeps on the FP32 pipes);
//   2. its right rotations W32, widened to df64, re-orthogonalised by one
//      Newton-Schulz step W <- W (3I - W^T W) / 2 (quadratic: 1e-7 -> 1e-14);
//   3. A = B W in df64.
// k_small_svd then finishes with df64 sweeps from (A, W), which converge in
// about two sweeps because A's columns are already nearly orthogonal.
// T1 is a c x c df64 scratch array.
template <int THREADS>
SSA_D void svd_precondition_body(const df64* __restrict__ B, int ldb, int r, int c, df64* __restrict__ A,
                                 df64* __restrict__ W, df64* __restrict__ T1, int cc, int max_sweeps, float tol32,
                                 float* A32 /* r x c, shared */, float* W32 /* c x c, shared */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = THREADS / 32;
  __shared__ int rotated;
  for (int e = threadIdx.x; e < r * c; e += THREADS) {
    const int i = e % r, j = e / r;
    const df64 b = B[(int64_t)i * ldb + j];
    A32[j * r + i] = b.hi + b.lo;
  }
  for (int e = threadIdx.x; e < c * c; e += THREADS) W32[e] = (e % c == e / c) ? 1.f : 0.f;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < cc - 1; ++rnd) {
      for (int pr = warp; pr < cc / 2; pr += nw) {
        const int2 pq = rr_pair(rnd, pr, cc);
        const int p = pq.x, q = pq.y;
        if (p >= c || q >= c) continue;
        float* ap = A32 + p * r;
        float* aq = A32 + q * r;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < r; i += 32) {
          const float x = ap[i], y = aq[i];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
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
        for (int i = lane; i < r; i += 32) {
          const float x = ap[i], y = aq[i];
          ap[i] = cs * x - sn * y;
          aq[i] = sn * x + cs * y;
        }
        float* wp = W32 + p * c;
        float* wq = W32 + q * c;
        for (int i = lane; i < c; i += 32) {
          const float x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // T1 = W32^T W32 (exact products of floats, df64 sums); W = W32 (1.5 I - 0.5 T1)
  for (int e = threadIdx.x; e < c * c; e += THREADS) {
    const int i = e % c, j = e / c;
    const float* wi = W32 + i * c;
    const float* wj = W32 + j * c;
    df64 a = df_zero();
    for (int k = 0; k < c; ++k) a = df_add(a, two_prod(wi[k], wj[k]));
    T1[(int64_t)j * c + i] = a;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * c; e += THREADS) {
    const int row = e % c, j = e / c;
    df64 a = df_zero();
    for (int i = 0; i < c; ++i) a = df_fma(make_df(W32[i * c + row], 0.f), T1[(int64_t)j * c + i], a);
    const df64 wkj = make_df(W32[j * c + row], 0.f);
    W[(int64_t)j * c + row] = df_sub(df_mul_f(wkj, 1.5f), df_scale(a, 0.5f));
  }
  __syncthreads();
  // The FP32 rotations are orthogonal to about 1e-5 and one step leaves about
  // 1e-10: a second Newton-Schulz step in df64 brings W to df64 rounding, so
  // the right Ritz vectors V Q stay unit vectors.  T1 = W^T W; A = W (1.5 I -
  // 0.5 T1) (A is at least c x c); W = A.
  for (int e = threadIdx.x; e < c * c; e += THREADS) {
    const int i = e % c, j = e / c;
    const df64* wi = W + (int64_t)i * c;
    const df64* wj = W + (int64_t)j * c;
    df64 a = df_zero();
    for (int k = 0; k < c; ++k) a = df_fma(wi[k], wj[k], a);
    T1[(int64_t)j * c + i] = a;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * c; e += THREADS) {
    const int row = e % c, j = e / c;
    df64 a = df_zero();
    for (int i = 0; i < c; ++i) a = df_fma(W[(int64_t)i * c + row], T1[(int64_t)j * c + i], a);
    A[(int64_t)j * c + row] = df_sub(df_mul_f(W[(int64_t)j * c + row], 1.5f), df_scale(a, 0.5f));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * c; e += THREADS) W[e] = A[e];
  __syncthreads();
  // A = B[:r, :c] W (df64)
  for (int e = threadIdx.x; e < r * c; e += THREADS) {
    const int i = e % r, j = e / r;
    df64 a = df_zero();
    for (int k = 0; k < c; ++k) a = df_fma(B[(int64_t)i * ldb + k], W[(int64_t)j * c + k], a);
    A[(int64_t)j * r + i] = a;
  }
}


}  // namespace ssa
