// Heterogeneity matrix (section 6.4) on the GPU.
//
// g_ij = 1 - sum_{t in test j} sum_{l in I} (U_{i,l}^T X_t)^2 / sum_{t in test j} ||X_t||^2
// where U_{i,l} are left singular vectors of base subseries i and X_t the
// L-lagged vectors.  The lagged vectors of test subseries j are the columns
// t = j .. j+T-L of the L-trajectory matrix X of the whole series, so one
// Algorithm 3 product X^T U_{i,l} of the whole series gives U_{i,l}^T X_t for
// every test window at once; the window sums come from prefix sums.
//   1. all base decompositions: batched launches (one persistent kernel over
//      the sliding windows), or one plan reused for every window when B
//      exceeds the batched engine's limits;
//   2. the selected vectors of a chunk of bases gathered into one block and
//      multiplied by X^T in one call;
//   3. per base one CTA: s(t) = sum_l y_l(t)^2, its prefix sums, and g_ij for
//      every test window against the prefix sums of ||X_t||^2.
// Prefix sums and window differences run in native FP64: they are O(N) per
// base, far below the products, and IEEE double keeps the cancellation of
// the window differences at 1e-16 relative to the prefix totals.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ssa.h"
#include "budget.h"
#include "prof.h"

using ssa::host_set_error;

namespace {

constexpr int HT = 512;

// out[i * B + t] = f[i0 + i + t]: the sliding base windows of a chunk
__global__ void k_gather_windows(const double* __restrict__ f, int64_t i0, int64_t B, int64_t count,
                                 double* __restrict__ out) {
  const int64_t tot = count * B;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / B, t = e - i * B;
    out[e] = f[i0 + i + t];
  }
}

// inclusive block scan of one value per thread (512 threads)
__device__ double block_scan(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = lane < HT / 32 ? red[lane] : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < HT / 32) red[lane] = w;
  }
  __syncthreads();
  const double before = warp ? red[warp - 1] : 0.0;
  __syncthreads();
  return v + before;
}

// P[0] = 0, P[t+1] = P[t] + val(t) for t < n: one CTA, segments of n/HT per thread
template <class F>
__device__ void block_prefix(int64_t n, F val, double* __restrict__ P, double* red) {
  const int64_t seg = (n + HT - 1) / HT;
  const int64_t a = threadIdx.x * seg, b = std::min<int64_t>(n, a + seg);
  double s = 0.0;
  for (int64_t t = a; t < b; ++t) s += val(t);
  const double incl = block_scan(s, red);
  double run = incl - s;
  if (threadIdx.x == 0) P[0] = 0.0;
  for (int64_t t = a; t < b; ++t) {
    run += val(t);
    P[t + 1] = run;
  }
}

// Pq: prefix sums of q(t) = ||X_t||^2 = sum_{m=t}^{t+L-1} f_m^2 (one CTA);
// Pf is scratch for the prefix sums of f^2 (N + 1).
__global__ void __launch_bounds__(HT) k_lag_norms(const double* __restrict__ f, int64_t N, int64_t L,
                                                  double* __restrict__ Pf, double* __restrict__ Pq) {
  __shared__ double red[HT / 32];
  block_prefix(N, [&](int64_t t) { return f[t] * f[t]; }, Pf, red);
  __syncthreads();
  const int64_t K = N - L + 1;
  block_prefix(K, [&](int64_t t) { return Pf[t + L] - Pf[t]; }, Pq, red);
}

// One CTA per base of the chunk: Y holds nI products X^T U_{i,l} per base
// (length K each); row i0 + b of H gets g for every test window.
__global__ void __launch_bounds__(HT) k_hrows(const double* __restrict__ Y, int nI, int64_t K, int64_t T, int64_t L,
                                              int64_t ntest, const double* __restrict__ Pq,
                                              double* __restrict__ Ps_all, double* __restrict__ H, int64_t ldh) {
  __shared__ double red[HT / 32];
  const int64_t b = blockIdx.x;
  const double* y = Y + b * nI * K;
  double* Ps = Ps_all + b * (K + 1);
  block_prefix(K, [&](int64_t t) {
    double s = 0.0;
    for (int l = 0; l < nI; ++l) {
      const double v = y[(int64_t)l * K + t];
      s = fma(v, v, s);
    }
    return s;
  }, Ps, red);
  __syncthreads();
  const int64_t w = T - L + 1;  // lagged vectors per test window
  double* row = H + b * ldh;
  for (int64_t j = threadIdx.x; j < ntest; j += HT) {
    const double den = Pq[j + w] - Pq[j];
    const double num = Ps[j + w] - Ps[j];
    double g = den > 0.0 ? (den - num) / den : 0.0;
    row[j] = g < 0.0 ? 0.0 : (g > 1.0 ? 1.0 : g);
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(size_t bytes, cudaStream_t st) {
    s = st;
    return cudaMallocAsync(&p, bytes, st);
  }
  template <class T> T* as() { return static_cast<T*>(p); }
};

}  // namespace

#define HK(x)                                                           \
  do {                                                                  \
    cudaError_t e_ = (x);                                               \
    if (e_ != cudaSuccess) {                                            \
      char m_[256];                                                     \
      std::snprintf(m_, sizeof m_, "%s: %s", #x, cudaGetErrorString(e_)); \
      host_set_error(m_);                                               \
      return e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA;  \
    }                                                                   \
  } while (0)

extern "C" int ssa_hmatrix(const double* f, int64_t N, int64_t L, int64_t B, int64_t T, const int32_t* I, int nI,
                           const ssa_opts_t* opts, double* H) {
  if (!f || !I || !H || nI < 1) {
    host_set_error("NULL argument or empty index set");
    return SSA_EINVAL;
  }
  if (!(1 < L && L < B && B <= N && L <= T && T <= N)) {
    host_set_error("need 1 < L < B <= N and L <= T <= N");
    return SSA_EINVAL;
  }
  const int64_t Kb = B - L + 1;
  const int64_t rmax = std::min(L, Kb);
  int kmax = 0;
  for (int a = 0; a < nI; ++a) {
    if (I[a] < 1 || I[a] > rmax) {
      host_set_error("index set entries must lie in 1..min(L, B-L+1)");
      return SSA_EINVAL;
    }
    for (int c = 0; c < a; ++c)
      if (I[c] == I[a]) {
        host_set_error("index set entries must be distinct");
        return SSA_EINVAL;
      }
    kmax = std::max(kmax, (int)I[a]);
  }
  ssa_opts_t o;
  if (opts) o = *opts;
  else ssa_default_opts(&o);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o.stream);
  const int64_t nb = N - B + 1, nt = N - T + 1, K = N - L + 1;
  // series on the device
  DevBuf fbuf;
  const double* fd = f;
  if (!on_device(f)) {
    HK(fbuf.alloc(N * sizeof(double), s));
    HK(cudaMemcpyAsync(fbuf.p, f, N * sizeof(double), cudaMemcpyHostToDevice, s));
    fd = fbuf.as<double>();
  }
  // prefix sums of the lagged-vector norms
  DevBuf Pf, Pq;
  HK(Pf.alloc((N + 1) * sizeof(double), s));
  HK(Pq.alloc((K + 1) * sizeof(double), s));
  k_lag_norms<<<1, HT, 0, s>>>(fd, N, L, Pf.as<double>(), Pq.as<double>());
  HK(cudaGetLastError());
  // plan of the whole series for the products X^T u
  ssa_plan_t plan = nullptr;
  int rc = ssa_embed_plan(N, L, &o, &plan);
  if (rc) return rc;
  struct PlanGuard {
    ssa_plan_t p;
    ~PlanGuard() { ssa_plan_destroy(p); }
  } pg{plan};
  rc = ssa_set_series(plan, fd);
  if (rc) return rc;
  int64_t M = 4;
  while (M < N) M *= 2;
  const bool batched = ssa::batch_eligible(B, L, kmax, o.precision);
  // chunk of bases: windows, vectors and products within ~1 GiB
  const int64_t per_base = B * 8 + L * kmax * 8 + nI * (L + K) * 8 + (K + 1) * 8 +
                           (M >= 32768 ? nI * (M / 2) * 16 : 0);
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nb, ((int64_t)1 << 30) / per_base));
  if (batched) chunk = std::min<int64_t>(chunk, 8192);
  DevBuf win, Ub, X, Y, Ps, Hd;
  HK(win.alloc(chunk * B * sizeof(double), s));
  HK(Ub.alloc(chunk * L * kmax * sizeof(double), s));
  HK(X.alloc(chunk * nI * L * sizeof(double), s));
  HK(Y.alloc(chunk * nI * K * sizeof(double), s));
  HK(Ps.alloc(chunk * (K + 1) * sizeof(double), s));
  const bool hdev = on_device(H);
  if (!hdev) HK(Hd.alloc(chunk * nt * sizeof(double), s));
  // one plan reused for every base window when the batched engine does not apply
  ssa_plan_t bplan = nullptr;
  if (!batched) {
    rc = ssa_embed_plan(B, L, &o, &bplan);
    if (rc) return rc;
  }
  struct PlanGuard2 {
    ssa_plan_t p;
    ~PlanGuard2() {
      if (p) ssa_plan_destroy(p);
    }
  } pg2{bplan};
  int worst = SSA_OK;
  std::vector<int64_t> off, Ls;
  std::vector<int32_t> ks;
  for (int64_t i0 = 0; i0 < nb; i0 += chunk) {
    const int64_t cnt = std::min(chunk, nb - i0);
    double* U = Ub.as<double>();
    if (batched) {
      k_gather_windows<<<(int)std::min<int64_t>(4096, (cnt * B + 255) / 256), 256, 0, s>>>(fd, i0, B, cnt,
                                                                                         win.as<double>());
      HK(cudaGetLastError());
      off.assign(cnt + 1, 0);
      for (int64_t i = 0; i < cnt; ++i) off[i + 1] = off[i] + B;
      Ls.assign(cnt, L);
      ks.assign(cnt, kmax);
      ssa_batch_t b = nullptr;
      rc = ssa_decompose_batch((int)cnt, win.as<double>(), off.data(), Ls.data(), ks.data(), &o, &b);
      if (rc != SSA_OK && rc != SSA_ENOCONV) return rc;
      if (rc == SSA_ENOCONV) worst = SSA_ENOCONV;
      // the batch's left vectors are already laid out base after base (L x kmax each)
      HK(cudaMemcpyAsync(U, ssa::batch_device_U(b), cnt * L * kmax * sizeof(double), cudaMemcpyDeviceToDevice, s));
      ssa_batch_destroy(b);
    } else {
      for (int64_t i = 0; i < cnt; ++i) {
        ssa_decomp_t d = nullptr;
        rc = ssa_decompose(bplan, fd + i0 + i, kmax, &d);
        if (rc != SSA_OK && rc != SSA_ENOCONV) return rc;
        if (rc == SSA_ENOCONV) worst = SSA_ENOCONV;
        rc = ssa_decomp_get(d, nullptr, U + i * L * kmax, nullptr, nullptr);
        ssa_decomp_destroy(d);
        if (rc) return rc;
      }
    }
    // selected vectors: X[i][m] = U_i[:, I[m] - 1]
    for (int m = 0; m < nI; ++m)
      HK(cudaMemcpy2DAsync(X.as<double>() + m * L, nI * L * sizeof(double), U + (int64_t)(I[m] - 1) * L,
                           L * kmax * sizeof(double), L * sizeof(double), cnt, cudaMemcpyDeviceToDevice, s));
    // products X^T U for the whole series (Algorithm 3), all vectors of the chunk in one call
    rc = ssa_matvec(plan, 1, X.as<double>(), Y.as<double>(), (int)(cnt * nI));
    if (rc) return rc;
    double* Hout = hdev ? H + i0 * nt : Hd.as<double>();
    k_hrows<<<(int)cnt, HT, 0, s>>>(Y.as<double>(), nI, K, T, L, nt, Pq.as<double>(), Ps.as<double>(), Hout, nt);
    HK(cudaGetLastError());
    if (!hdev) HK(cudaMemcpyAsync(H + i0 * nt, Hd.p, cnt * nt * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  HK(cudaStreamSynchronize(s));
  if (worst == SSA_ENOCONV) host_set_error("a base decomposition did not converge within max_restarts");
  return worst;
}
