// ssa_matvec_noalloc: the trajectory-matrix product (spectrum of the series,
// then X x or X^T x) without any device allocation.  Its working memory --
// the spectrum, the four-step scratch and the twiddle tables -- is a
// file-scope __device__ array of fixed size, so the entry point can serve
// callers that may not allocate device memory (see include/ssa.h).
#include <cmath>
#include <cstdio>
#include <mutex>

#include "ssa.h"
#include "spectral.h"
#include "prof.h"

using namespace ssa;

namespace {

constexpr int64_t NA_MAX_N = 65536;               // largest series (FFT length M <= 65536)
constexpr int64_t NA_MAX_HALF = NA_MAX_N / 2;     // n = M / 2 complex points
constexpr int64_t NA_TW = 16384;                  // largest direct twiddle table (single-CTA FP32 path)
constexpr int64_t NA_TWO = 256;                   // each half of the two-level W_M table
constexpr int64_t NA_CHAT = NA_MAX_HALF + 1;      // spectrum C_0..C_n
constexpr int64_t NA_TOTAL = NA_CHAT + NA_MAX_HALF + NA_TW + 2 * NA_TWO;

constexpr int na_lg(int64_t x) { return x <= 1 ? 0 : 1 + na_lg(x / 2); }
// the largest tables a series of up to NA_MAX_N needs fit their slots: the
// single-CTA FP32 product at n = 16384 uses W_n directly, a four-step product
// W_{n2} with n2 <= n; the two-level W_M table halves are M >> tws and 2^tws
static_assert(SMALL_MAXE_F32 <= NA_TW && SMALL_MAXE_DF64 <= NA_TW, "direct twiddle slot too small");
static_assert((NA_MAX_N >> ((na_lg(NA_MAX_N) + 1) / 2)) <= NA_TWO, "two-level table slot too small");
static_assert(((int64_t)1 << ((na_lg(NA_MAX_N) + 1) / 2)) <= NA_TWO, "two-level table slot too small");

// Shared by every call in the process, on every device that loads the library.
static __device__ __align__(256) cplx<df64> g_na_scratch[NA_TOTAL];

constexpr int NA_MAX_DEV = 64;
static void* g_na_addr[NA_MAX_DEV];
static std::mutex g_na_mu;

int fail(int code, const char* msg) {
  host_set_error(msg);
  return code;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// W_P^m = exp(-2 pi i m / P) in df64; 2m/P is exact, so sincospi sees an exact argument.
__device__ cplx<df64> na_twiddle(int64_t m, int64_t P) {
  double sn, cs;
  sincospi(2.0 * (double)m / (double)P, &sn, &cs);
  cplx<df64> z;
  z.re = df_from_double(cs);
  z.im = df_from_double(-sn);
  return z;
}

__global__ void k_na_twiddles(cplx<df64>* tw, int64_t P, cplx<df64>* tA, int64_t nA, int tws, cplx<df64>* tB,
                              int64_t nB, int64_t M) {
  const int64_t total = P + nA + nB;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < P) tw[i] = na_twiddle(i, P);
    else if (i < P + nA) tA[i - P] = na_twiddle((i - P) << tws, M);
    else tB[i - P - nA] = na_twiddle(i - P - nA, M);
  }
}

// Device address of the scratch array on the current device, looked up
// once per device (the host-side name is only a stand-in for it).
int scratch_address(cplx<df64>** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SSA_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEV) return fail(SSA_EINVAL, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      char msg[256];
      std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
      return fail(SSA_ECUDA, msg);
    }
    g_na_addr[dev] = p;
  }
  *out = static_cast<cplx<df64>*>(g_na_addr[dev]);
  return SSA_OK;
}

struct SuppressProf {
  SuppressProf() { prof_suppress(true); }
  ~SuppressProf() { prof_suppress(false); }
};

}  // namespace

extern "C" int ssa_matvec_noalloc(const double* f, int64_t N, int64_t L, int transpose, const double* x, double* y,
                                  int precision, void* stream) {
  if (!f || !x || !y) return fail(SSA_EINVAL, "NULL argument");
  if (N <= 2 || L <= 1 || L >= N) return fail(SSA_EINVAL, "need N > 2 and 1 < L < N");
  if (N > NA_MAX_N) return fail(SSA_EINVAL, "ssa_matvec_noalloc supports N <= 65536 (fixed scratch size); use a plan");
  if (precision != SSA_PREC_F64 && precision != SSA_PREC_F32C) return fail(SSA_EINVAL, "unknown precision");
  if (!on_device(f) || !on_device(x) || !on_device(y))
    return fail(SSA_EINVAL, "ssa_matvec_noalloc needs device pointers (it cannot stage host buffers)");
  cplx<df64>* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SuppressProf guard;
  // geometry, as ssa_embed_plan chooses it
  const int64_t K = N - L + 1;
  const bool transposed = L > K;
  int64_t M = 4;
  while (M < N) M *= 2;
  Geom g{};
  g.N = N;
  g.L = transposed ? K : L;
  g.K = transposed ? L : K;
  g.M = M;
  int lgM = 0;
  while (((int64_t)1 << lgM) < M) ++lgM;
  g.lg_n = lgM - 1;
  g.lg_n1 = g.lg_n / 2;
  g.lg_n2 = g.lg_n - g.lg_n1;
  const bool small = small_path(g, precision);
  g.lg_P = small ? g.lg_n : g.lg_n2;
  g.tws = (lgM + 1) / 2;
  g.twshift = 0;
  const int64_t n = (int64_t)1 << g.lg_n, P = (int64_t)1 << g.lg_P;
  const int64_t nA = M >> g.tws, nB = (int64_t)1 << g.tws;
  // carve the array: spectrum | four-step scratch | W_P | tA | tB
  cplx<df64>* chat = scratch;
  cplx<df64>* Y = chat + NA_CHAT;
  cplx<df64>* tw = Y + NA_MAX_HALF;
  cplx<df64>* tA = tw + NA_TW;
  cplx<df64>* tB = tA + NA_TWO;
  if (P > NA_TW || nA > NA_TWO || nB > NA_TWO || n > NA_MAX_HALF)
    return fail(SSA_EINVAL, "ssa_matvec_noalloc: table sizes exceed the fixed scratch layout");
  g.tw = tw;
  g.tA = tA;
  g.tB = tB;
  k_na_twiddles<<<64, 256, 0, s>>>(tw, P, tA, nA, g.tws, tB, nB, M);
  // every part of the array that is read is written first in this call, so
  // nothing needs clearing between calls
  launch_spectrum(g, f, chat, small ? 1 : 0, 1.0f / (4.0f * (float)n), Y, s);
  const int t = (transpose ? 1 : 0) ^ (transposed ? 1 : 0);
  const int64_t in_len = t ? g.L : g.K, out_len = t ? g.K : g.L;
  launch_matvec_d(g, precision, t, x, in_len, y, out_len, 1, chat, Y, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SSA_ECUDA, cudaGetErrorString(e));
  return SSA_OK;
}
