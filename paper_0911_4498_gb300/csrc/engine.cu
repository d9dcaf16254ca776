// Host engine and C ABI (include/ssa.h): plans, the spectrum of the series,
// batched trajectory-matrix products, the thick-restart Golub-Kahan-Lanczos
// driver (section 3) and grouped Hankelization (section 5).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "ssa.h"
#include "budget.h"
#include "lanczos.h"
#include "spectral.h"
#include "prof.h"

using namespace ssa;

// ------------------------------------------------------------------ errors
static thread_local char g_err[512];
static void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
namespace ssa {
// detail message for ssa_last_error(), for the other translation units
void host_set_error(const char* msg) { std::snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace ssa
#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      set_err("%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA;         \
    }                                                                           \
  } while (0)
#define CHECK_LAUNCH() CK(cudaGetLastError())
#define REQ(cond, ...)           \
  do {                           \
    if (!(cond)) {               \
      set_err(__VA_ARGS__);      \
      return SSA_EINVAL;         \
    }                            \
  } while (0)

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host-side fault injection for tests (ssa_fault_inject_alloc): when armed
// with n >= 0, the next n device allocations of this file succeed and the one
// after them fails as if the device were out of memory, without calling the
// allocator; then the injection disarms itself.
static std::atomic<int64_t> g_fail_after{-1};
// The library's stream-ordered allocations come from its own memory pool on each device, which
// keeps up to 4 GiB of freed memory for reuse.  The device's default pool hands freed memory
// back to the CUDA driver at every synchronisation, so the per-call scratch of the reconstruction
// (about 1.3 GB at N = 2^20) and host-output staging were mapped again on every call.
static cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  static bool tried[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!tried[dev]) {
    tried[dev] = true;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
      uint64_t keep = (uint64_t)4 << 30;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      pools[dev] = pool;
    } else {
      cudaGetLastError();  // fall back to the default pool
    }
  }
  return pools[dev];
}

namespace ssa {
void lib_pool_keep(uint64_t bytes) {
  cudaMemPool_t pool = lib_pool();
  if (!pool) return;
  uint64_t cur = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && bytes > cur)
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &bytes);
  cudaGetLastError();
}
}  // namespace ssa

template <class T> static cudaError_t dev_alloc(T** ptr, size_t bytes, cudaStream_t s) {
  int64_t v = g_fail_after.load();
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1)) {
      if (v == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  cudaMemPool_t pool = lib_pool();
  if (pool) return cudaMallocFromPoolAsync(reinterpret_cast<void**>(ptr), bytes, pool, s);
  return cudaMallocAsync(reinterpret_cast<void**>(ptr), bytes, s);
}

// Device view of a caller buffer: host buffers are staged through a
// stream-ordered allocation (returned to the pool on release).
template <class T>
struct Staged {
  T* dev = nullptr;
  T* owned = nullptr;
  const T* host_src = nullptr;
  T* host_dst = nullptr;
  size_t count = 0;
  cudaStream_t s = nullptr;
  int in(const T* p, size_t n, cudaStream_t st) {
    s = st;
    count = n;
    if (is_device_ptr(p)) {
      dev = const_cast<T*>(p);
      return SSA_OK;
    }
    CK(dev_alloc(&owned, n * sizeof(T) + 16, st));
    CK(cudaMemcpyAsync(owned, p, n * sizeof(T), cudaMemcpyHostToDevice, st));
    dev = owned;
    return SSA_OK;
  }
  int out(T* p, size_t n, cudaStream_t st) {
    s = st;
    count = n;
    if (is_device_ptr(p)) {
      dev = p;
      return SSA_OK;
    }
    CK(dev_alloc(&owned, n * sizeof(T) + 16, st));
    dev = owned;
    host_dst = p;
    return SSA_OK;
  }
  int finish() {
    if (host_dst) CK(cudaMemcpyAsync(host_dst, dev, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    return SSA_OK;
  }
  bool needs_sync() const { return host_dst != nullptr; }
  ~Staged() {
    if (owned) cudaFreeAsync(owned, s);
  }
};

// ------------------------------------------------------------------ tables
// (cos, sin) of 2 pi m / P, reduced to the first octant so the double
// cos/sin are evaluated on |theta| <= pi/4.
static void cis_turn(int64_t m, int64_t P, double& c, double& s) {
  m %= P;
  if (m < 0) m += P;
  if (P % 8 != 0) {
    const double th = 2.0 * M_PI * (double)m / (double)P;
    c = std::cos(th);
    s = std::sin(th);
    if (P == 1 || m == 0) { c = 1; s = 0; }
    if (P == 2 && m == 1) { c = -1; s = 0; }
    if (P == 4) {
      const double cc[4] = {1, 0, -1, 0}, ss[4] = {0, 1, 0, -1};
      c = cc[m];
      s = ss[m];
    }
    return;
  }
  const int64_t q = P / 4;
  const int quad = (int)(m / q);
  int64_t rr = m - quad * q;  // angle within the quadrant, [0, P/4)
  double c0, s0;
  if (2 * rr <= q) {
    const double th = 2.0 * M_PI * (double)rr / (double)P;
    c0 = std::cos(th);
    s0 = std::sin(th);
  } else {
    const double th = 2.0 * M_PI * (double)(q - rr) / (double)P;
    c0 = std::sin(th);
    s0 = std::cos(th);
  }
  switch (quad) {
    case 0: c = c0; s = s0; break;
    case 1: c = -s0; s = c0; break;
    case 2: c = -c0; s = -s0; break;
    default: c = s0; s = -c0; break;
  }
}

static cplx<df64> tw_entry(int64_t m, int64_t P) {
  double c, s;
  cis_turn(m, P, c, s);
  cplx<df64> z;
  z.re = df_from_double(c);
  z.im = df_from_double(-s);  // W_P^m = exp(-2 pi i m / P)
  return z;
}

static cplx<double> tw_entry64(int64_t m, int64_t P) {
  double c, s;
  cis_turn(m, P, c, s);
  return mk(c, -s);
}

static int ilog2(int64_t x) {
  int r = 0;
  while (((int64_t)1 << r) < x) ++r;
  return r;
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// plan's stream): creating and destroying plans and decompositions never
// synchronises the device, so requests on other streams keep running.
static void free_async(void* ptr, cudaStream_t s) {
  if (ptr) cudaFreeAsync(ptr, s);
}
template <class T> static cudaError_t malloc_async(T** ptr, size_t bytes, cudaStream_t s) {
  return dev_alloc(ptr, bytes, s);
}

// ------------------------------------------------------------------ handles
struct Workspace {
  int dcap = 0;
  int64_t ldu = 0, ldv = 0;
  df64* Ub[2] = {nullptr, nullptr};
  df64* Vb[2] = {nullptr, nullptr};
  df64* B = nullptr;
  int ldb = 0;
  df64* y = nullptr;
  ReorthWork rw{};
  SvdWork sw{};
  SvdWork sw2{};  // ghost filtering: the projected matrix without its first row
  df64* est = nullptr;
  df64* dummy = nullptr;
  int* flag = nullptr;
  unsigned* status = nullptr;
  int* sgn = nullptr;
  ProState pro{};
  void release(cudaStream_t st) {
    free_async(pro.M, st);
    free_async(pro.N, st);
    free_async(pro.force, st);
    pro = ProState{};
    for (int i = 0; i < 2; ++i) {
      free_async(Ub[i], st);
      free_async(Vb[i], st);
      Ub[i] = Vb[i] = nullptr;
    }
    free_async(B, st);
    free_async(y, st);
    free_async(rw.part, st);
    free_async(rw.part2, st);
    free_async(rw.coop, st);
    free_async(rw.h, st);
    free_async(rw.h2, st);
    free_async(rw.gate, st);
    free_async(rw.run, st);
    free_async(rw.skip, st);
    free_async(rw.nrm, st);
    free_async(rw.counter, st);
    for (SvdWork* v : {&sw2}) {
      free_async(v->A, st);
      free_async(v->W, st);
      free_async(v->sigma, st);
      free_async(v->P, st);
      free_async(v->Q, st);
      free_async(v->resid, st);
      free_async(v->sigma_d, st);
      free_async(v->conv, st);
      *v = SvdWork{};
    }
    free_async(sw.A, st);
    free_async(sw.W, st);
    free_async(sw.sigma, st);
    free_async(sw.P, st);
    free_async(sw.Q, st);
    free_async(sw.resid, st);
    free_async(sw.sigma_d, st);
    free_async(sw.conv, st);
    free_async(est, st);
    free_async(dummy, st);
    free_async(flag, st);
    free_async(status, st);
    free_async(sgn, st);
    B = y = est = dummy = nullptr;
    rw = ReorthWork{};
    sw = SvdWork{};
    flag = nullptr;
    status = nullptr;
    sgn = nullptr;
    dcap = 0;
  }
};

struct ssa_plan_s {
  int64_t N = 0, L = 0, K = 0, Lw = 0, Kw = 0;
  bool transposed = false;
  ssa_opts_t opts{};
  cudaStream_t stream = nullptr;
  Geom g{};
  bool small = false;
  cplx<df64>* tw = nullptr;
  cplx<df64>* tA = nullptr;
  cplx<df64>* tB = nullptr;
  cplx<df64>* chat = nullptr;
  void* scratch = nullptr;
  double* f_dev = nullptr;
  // IEEE-double tables and spectrum for the Rayleigh-quotient refinement (made on first use)
  cplx<double>* tw64 = nullptr;
  cplx<double>* tA64 = nullptr;
  cplx<double>* tB64 = nullptr;
  cplx<double>* chat64 = nullptr;
  bool has_series = false;
  // The series is held scaled by 2^-fexp (max |f| in [1/2, 1)), an exact
  // change of units that keeps every double-float quantity of the method far
  // from FP32's overflow and underflow; sigma, residuals and products are
  // scaled back by 2^fexp (U, V do not change, and Hankelization with the
  // returned sigma is in the caller's units).
  int fexp = 0;
  unsigned long long* fstat = nullptr;  // device: [0] max |f| (bits), [1] non-finite count
  Workspace ws;
  // CUDA graphs of whole Lanczos cycles (the half-steps between two convergence tests), keyed by
  // their shape; a shape is captured when it runs again in a later decomposition with this
  // workspace (restart cycles repeat shapes within one decomposition, and a graph captured there
  // would be replayed once or twice at most), so that a plan used once pays no capture
  int64_t lanczos_calls = 0;
  struct CycleGraph {
    int cur, r0, c0, d;
    bool pro, none;
    int64_t first_call;
    bool captured, failed;
    cudaGraphExec_t exec;
    int dr, dc;
    int64_t dmv;
    uint64_t launches;
  };
  std::vector<CycleGraph> cycles;
  void drop_cycles() {
    for (auto& e : cycles)
      if (e.exec) cudaGraphExecDestroy(e.exec);
    cycles.clear();
  }
};

struct ssa_decomp_s {
  ssa_plan_t plan = nullptr;
  int k = 0, d = 0, converged = 0, restarts = 0;
  int64_t matvecs = 0;
  double* sigma = nullptr;  // k
  double* resid = nullptr;  // k
  double* U = nullptr;      // L x k (user orientation)
  double* V = nullptr;      // K x k
  df64* Uw = nullptr;       // Lw x k (working orientation, for Hankelization)
  df64* Vw = nullptr;       // Kw x k
};


// ------------------------------------------------------------------ launch stats
namespace ssa {
static const char* const kClassNames[K_NCLASS] = {
    "spectrum", "matvec_small", "matvec_colfwd", "matvec_row", "matvec_colinv", "cgs_proj", "cgs_update",
    "cgs_update_proj", "normalize", "small_svd", "svd_precondition", "ritz", "hankel_small", "hankel_fourstep",
    "misc", "skipped", "batch_ssa"};
struct PendingLaunch {
  int cls;
  cudaEvent_t a, b;
  double bytes, flops;
  int launches;
};
struct ClassAcc {
  uint64_t launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};
static std::mutex g_pmu;
static bool g_pon = false;
static std::atomic<uint64_t> g_launches{0};
static std::vector<PendingLaunch> g_pending;
static std::vector<cudaEvent_t> g_evpool;
static ClassAcc g_acc[K_NCLASS];
static thread_local cudaEvent_t g_begin = nullptr;
static thread_local bool g_psup = false;
void prof_suppress(bool on) { g_psup = on; }

static cudaEvent_t ev_get() {
  if (!g_evpool.empty()) {
    cudaEvent_t e = g_evpool.back();
    g_evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
bool prof_enabled() { return g_pon; }
static thread_local uint64_t t_launches = 0;
uint64_t prof_thread_launches() { return t_launches; }
void prof_add_launches(uint64_t n) {
  g_launches += n;
  t_launches += n;
}
void prof_sub_launches(uint64_t n) {
  g_launches -= n;
  t_launches -= n;
}
void prof_begin(cudaStream_t s) {
  if (!g_pon || g_psup) return;
  std::lock_guard<std::mutex> lk(g_pmu);
  g_begin = ev_get();
  cudaEventRecord(g_begin, s);
}
void prof_end(cudaStream_t s, int cls, double bytes, double flops, int launches) {
  g_launches += launches;
  t_launches += launches;
  if (!g_pon || g_psup || !g_begin) return;
  std::lock_guard<std::mutex> lk(g_pmu);
  cudaEvent_t e = ev_get();
  cudaEventRecord(e, s);
  g_pending.push_back({cls, g_begin, e, bytes, flops, launches});
  g_begin = nullptr;
}
void prof_flush() {
  std::lock_guard<std::mutex> lk(g_pmu);
  std::vector<PendingLaunch> keep;
  for (auto& pl : g_pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, pl.a, pl.b);
    if (e == cudaErrorNotReady) {
      cudaGetLastError();
      keep.push_back(pl);
      continue;
    }
    if (e == cudaSuccess) {
      ClassAcc& c = g_acc[pl.cls];
      c.launches += pl.launches;
      c.ms += ms;
      c.bytes += pl.bytes;
      c.flops += pl.flops;
    } else {
      cudaGetLastError();
    }
    g_evpool.push_back(pl.a);
    g_evpool.push_back(pl.b);
  }
  g_pending.swap(keep);
}
}  // namespace ssa

extern "C" int ssa_stats_enable(int on) {
  {
    std::lock_guard<std::mutex> lk(g_pmu);
    if (on) {
      for (auto& c : g_acc) c = ClassAcc{};
      for (auto& pl : g_pending) {
        g_evpool.push_back(pl.a);
        g_evpool.push_back(pl.b);
      }
      g_pending.clear();
    }
    g_pon = on != 0;
  }
  return SSA_OK;
}

extern "C" int ssa_stats_get(ssa_kernel_stat_t* out, int max, int* count) {
  CK(cudaDeviceSynchronize());
  prof_flush();
  std::lock_guard<std::mutex> lk(g_pmu);
  if (count) *count = K_NCLASS;
  for (int i = 0; i < K_NCLASS && i < max && out; ++i) {
    std::memset(&out[i], 0, sizeof out[i]);
    std::snprintf(out[i].name, sizeof out[i].name, "%s", kClassNames[i]);
    out[i].launches = g_acc[i].launches;
    out[i].ms = g_acc[i].ms;
    out[i].bytes = g_acc[i].bytes;
    out[i].flops = g_acc[i].flops;
  }
  return SSA_OK;
}

extern "C" uint64_t ssa_kernel_launches(void) { return g_launches.load(); }

extern "C" int ssa_fault_inject_alloc(int64_t after) {
  g_fail_after.store(after < 0 ? -1 : after);
  return SSA_OK;
}

extern "C" void ssa_default_opts(ssa_opts_t* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = SSA_PREC_F64;
  o->tol = 0.0;
  o->max_restarts = 200;
  o->krylov_dim = 0;
  o->keep = 0;
  o->seed = 0;
  o->stream = nullptr;
  o->refine = SSA_REFINE_OFF;
  o->reorth_skip = 0.0;
  o->reorth = SSA_REORTH_FULL;
  o->grid_cap = 0;
}

extern "C" const char* ssa_strerror(int code) {
  switch (code) {
    case SSA_OK: return "ok";
    case SSA_EINVAL: return "invalid argument";
    case SSA_ENOMEM: return "out of device memory";
    case SSA_ENOCONV: return "Lanczos did not converge within max_restarts";
    case SSA_ECUDA: return "CUDA error";
    case SSA_ENUMERIC: return "non-finite value";
    default: return "unknown status";
  }
}
extern "C" const char* ssa_last_error(void) { return g_err; }

extern "C" void ssa_plan_destroy(ssa_plan_t p) {
  if (!p) return;
  p->drop_cycles();
  p->ws.release(p->stream);
  free_async(p->tw, p->stream);
  free_async(p->tA, p->stream);
  free_async(p->tB, p->stream);
  free_async(p->chat, p->stream);
  free_async(p->scratch, p->stream);
  free_async(p->f_dev, p->stream);
  free_async(p->fstat, p->stream);
  free_async(p->tw64, p->stream);
  free_async(p->tA64, p->stream);
  free_async(p->tB64, p->stream);
  free_async(p->chat64, p->stream);
  delete p;
}

extern "C" int ssa_embed_plan(int64_t N, int64_t L, const ssa_opts_t* opts, ssa_plan_t* out) {
  REQ(out != nullptr, "out is NULL");
  *out = nullptr;
  REQ(N > 2, "need N > 2 (got %lld)", (long long)N);
  REQ(L > 1 && L < N, "need 1 < L < N (got L=%lld, N=%lld)", (long long)L, (long long)N);
  REQ(N <= ((int64_t)1 << 23), "N up to 2^23 is supported (got %lld)", (long long)N);
  ssa_opts_t o;
  if (opts) o = *opts;
  else ssa_default_opts(&o);
  REQ(o.precision == SSA_PREC_F64 || o.precision == SSA_PREC_F32C, "unknown precision %d", o.precision);
  REQ(o.refine == SSA_REFINE_OFF || o.refine == SSA_REFINE_ON, "unknown refine mode %d", o.refine);
  REQ(o.reorth_skip >= 0.0 && o.reorth_skip < 1e-3, "reorth_skip must be in [0, 1e-3) (got %g)", o.reorth_skip);
  REQ(o.reorth == SSA_REORTH_FULL || o.reorth == SSA_REORTH_PRO || o.reorth == SSA_REORTH_NONE,
      "unknown reorth mode %d", o.reorth);
  REQ(o.reorth == SSA_REORTH_FULL || o.precision == SSA_PREC_F64,
      "partial or no reorthogonalisation needs SSA_PREC_F64 (the FP32 products' error is above sqrt(eps))");
  REQ(o.grid_cap >= 0, "grid_cap must be >= 0 (got %d)", o.grid_cap);
  ssa_plan_s* p = new (std::nothrow) ssa_plan_s();
  if (!p) return SSA_ENOMEM;
  p->opts = o;
  p->stream = reinterpret_cast<cudaStream_t>(o.stream);
  p->N = N;
  p->L = L;
  p->K = N - L + 1;
  p->transposed = L > p->K;
  p->Lw = p->transposed ? p->K : L;
  p->Kw = p->transposed ? L : p->K;
  int64_t M = 4;
  while (M < N) M *= 2;
  Geom& g = p->g;
  g.N = N;
  g.L = p->Lw;
  g.K = p->Kw;
  g.M = M;
  g.lg_n = ilog2(M) - 1;
  g.lg_n1 = g.lg_n / 2;
  g.lg_n2 = g.lg_n - g.lg_n1;
  p->small = small_path(g, o.precision);
  g.lg_P = p->small ? g.lg_n : g.lg_n2;
  const int64_t P = (int64_t)1 << g.lg_P;
  const int lgM = ilog2(M);
  g.tws = (lgM + 1) / 2;
  const int64_t nA = M >> g.tws, nB = (int64_t)1 << g.tws;
  std::vector<cplx<df64>> htw(P), hA(nA), hB(nB);
  for (int64_t m = 0; m < P; ++m) htw[m] = tw_entry(m, P);
  for (int64_t m = 0; m < nA; ++m) hA[m] = tw_entry(m << g.tws, M);
  for (int64_t m = 0; m < nB; ++m) hB[m] = tw_entry(m, M);
  auto fail = [&](int code) {
    ssa_plan_destroy(p);
    return code;
  };
  const int64_t n = (int64_t)1 << g.lg_n;
#define PK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      set_err("%s: %s", #x, cudaGetErrorString(e_)); \
      return fail(e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA); \
    }                                           \
  } while (0)
  PK(malloc_async(&p->tw, P * sizeof(cplx<df64>), p->stream));
  PK(malloc_async(&p->tA, nA * sizeof(cplx<df64>), p->stream));
  PK(malloc_async(&p->tB, nB * sizeof(cplx<df64>), p->stream));
  PK(malloc_async(&p->chat, (n + 1) * sizeof(cplx<df64>), p->stream));
  PK(malloc_async(&p->scratch, spectral_scratch_bytes(g), p->stream));
  PK(malloc_async(&p->f_dev, N * sizeof(double), p->stream));
  PK(malloc_async(&p->fstat, 2 * sizeof(unsigned long long), p->stream));
  PK(cudaMemcpyAsync(p->tw, htw.data(), P * sizeof(cplx<df64>), cudaMemcpyHostToDevice, p->stream));
  PK(cudaMemcpyAsync(p->tA, hA.data(), nA * sizeof(cplx<df64>), cudaMemcpyHostToDevice, p->stream));
  PK(cudaMemcpyAsync(p->tB, hB.data(), nB * sizeof(cplx<df64>), cudaMemcpyHostToDevice, p->stream));
#undef PK
  g.tw = p->tw;
  g.tA = p->tA;
  g.tB = p->tB;
  if (!p->small) {  // pick the column tiling of the four-step passes for this n (once per process)
    const int e = autotune_fourstep(g, o.precision, p->stream);
    if (e != 0) {
      set_err("four-step tiling autotune: %s", cudaGetErrorString((cudaError_t)e));
      return fail(SSA_ECUDA);
    }
  }
  *out = p;
  return SSA_OK;
}

extern "C" int ssa_fft_tiling(int precision, int64_t N, int* cols_fwd, int* cols_inv) {
  REQ(cols_fwd != nullptr && cols_inv != nullptr, "NULL argument");
  REQ(N > 2, "need N > 2");
  int64_t M = 4;
  while (M < N) M *= 2;
  const int lg_n = ilog2(M) - 1;
  const int a = tuned_tiling(precision, lg_n, 0), b = tuned_tiling(precision, lg_n, 1);
  *cols_fwd = a >= 0 ? 1 << a : 0;
  *cols_inv = b >= 0 ? 1 << b : 0;
  return SSA_OK;
}

extern "C" int ssa_fft_threads(int precision, int64_t N, int* th_fwd, int* th_row, int* th_inv) {
  REQ(th_fwd != nullptr && th_row != nullptr && th_inv != nullptr, "NULL argument");
  REQ(N > 2, "need N > 2");
  int64_t M = 4;
  while (M < N) M *= 2;
  const int lg_n = ilog2(M) - 1;
  *th_fwd = tuned_threads(precision, lg_n, 0);
  *th_row = tuned_threads(precision, lg_n, 2);
  *th_inv = tuned_threads(precision, lg_n, 1);
  return SSA_OK;
}

extern "C" int ssa_plan_info(ssa_plan_t p, int64_t* M, int* single_cta) {
  REQ(p != nullptr, "plan is NULL");
  if (M) *M = p->g.M;
  if (single_cta) *single_cta = p->small ? 1 : 0;
  return SSA_OK;
}

// max |f| (as the bits of a non-negative double, which order like integers)
// and the number of non-finite entries
__global__ void k_absmax_finite(const double* __restrict__ f, int64_t n, unsigned long long* out) {
  unsigned long long m = 0ull, bad = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(f[i]);
    if (!(a <= 1.7976931348623157e308)) ++bad;  // NaN or infinity
    else m = max(m, (unsigned long long)__double_as_longlong(a));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(out, m);
    if (bad) atomicAdd(out + 1, bad);
  }
}
// x[i] *= s (s a power of two: exact)
__global__ void k_scale_d(double* __restrict__ x, int64_t n, double s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= s;
}
__global__ void k_scale_copy_d(const double* __restrict__ src, double* __restrict__ dst, int64_t n, double s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] * s;
}
static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(1024, (n + 255) / 256)); }
static void scale_copy(const double* src, double* dst, int64_t n, int e, cudaStream_t s) {
  if (e == 0 && src == dst) return;
  k_scale_copy_d<<<grid_for(n), 256, 0, s>>>(src, dst, n, std::ldexp(1.0, e));
}

static int set_series(ssa_plan_t p, const double* f) {
  double fmax = 0.0;
  if (is_device_ptr(f)) {
    CK(cudaMemcpyAsync(p->f_dev, f, p->N * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    unsigned long long st[2] = {0ull, 0ull};
    CK(cudaMemsetAsync(p->fstat, 0, sizeof st, p->stream));
    k_absmax_finite<<<grid_for(p->N), 256, 0, p->stream>>>(p->f_dev, p->N, p->fstat);
    CHECK_LAUNCH();
    CK(cudaMemcpyAsync(st, p->fstat, sizeof st, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (st[1]) {
      set_err("f has %llu non-finite entries", st[1]);
      return SSA_ENUMERIC;
    }
    std::memcpy(&fmax, &st[0], sizeof fmax);
  } else {
    for (int64_t i = 0; i < p->N; ++i) {
      if (!std::isfinite(f[i])) {
        set_err("f[%lld] is not finite", (long long)i);
        return SSA_ENUMERIC;
      }
      fmax = std::max(fmax, std::fabs(f[i]));
    }
    CK(cudaMemcpyAsync(p->f_dev, f, p->N * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  }
  int e = 0;
  if (fmax > 0.0) std::frexp(fmax, &e);  // fmax = m 2^e, m in [1/2, 1)
  p->fexp = e;
  if (e != 0) {
    k_scale_d<<<grid_for(p->N), 256, 0, p->stream>>>(p->f_dev, p->N, std::ldexp(1.0, -e));
    CHECK_LAUNCH();
  }
  const float scale = 1.0f / (4.0f * (float)((int64_t)1 << p->g.lg_n));
  launch_spectrum(p->g, p->f_dev, p->chat, p->small ? 1 : 0, scale, p->scratch, p->stream);
  CHECK_LAUNCH();
  p->has_series = true;
  return SSA_OK;
}

extern "C" int ssa_set_series(ssa_plan_t p, const double* f) {
  REQ(p != nullptr && f != nullptr, "plan or f is NULL");
  int rc = set_series(p, f);
  if (rc) return rc;
  CK(cudaStreamSynchronize(p->stream));
  return SSA_OK;
}

extern "C" int ssa_get_spectrum(ssa_plan_t p, double* re, double* im) {
  REQ(p != nullptr && re != nullptr && im != nullptr, "NULL argument");
  REQ(p->has_series, "no series set");
  const int64_t n = (int64_t)1 << p->g.lg_n;
  std::vector<cplx<df64>> h(n + 1);
  CK(cudaMemcpyAsync(h.data(), p->chat, (n + 1) * sizeof(cplx<df64>), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const double unscale = 4.0 * (double)n * std::ldexp(1.0, p->fexp);
  std::vector<double> hre(n + 1), him(n + 1);
  const int64_t n1 = (int64_t)1 << p->g.lg_n1, n2 = (int64_t)1 << p->g.lg_n2;
  for (int64_t k = 0; k <= n; ++k) {
    int64_t pos = k;
    if (!p->small && k < n) {
      const int64_t c = k % n1, e = k / n1;
      pos = c * n2 + e;
    }
    hre[k] = df_to_double(h[pos].re) * unscale;
    him[k] = df_to_double(h[pos].im) * unscale;
  }
  const bool dre = is_device_ptr(re), dim_ = is_device_ptr(im);
  if (dre) CK(cudaMemcpy(re, hre.data(), (n + 1) * sizeof(double), cudaMemcpyHostToDevice));
  else std::memcpy(re, hre.data(), (n + 1) * sizeof(double));
  if (dim_) CK(cudaMemcpy(im, him.data(), (n + 1) * sizeof(double), cudaMemcpyHostToDevice));
  else std::memcpy(im, him.data(), (n + 1) * sizeof(double));
  return SSA_OK;
}

extern "C" int ssa_matvec(ssa_plan_t p, int transpose, const double* x, double* y, int nvec) {
  REQ(p != nullptr && x != nullptr && y != nullptr, "NULL argument");
  REQ(nvec >= 1, "nvec must be >= 1");
  REQ(p->has_series, "no series set (ssa_set_series)");
  const int t = (transpose ? 1 : 0) ^ (p->transposed ? 1 : 0);
  const int64_t in_len = t ? p->Lw : p->Kw, out_len = t ? p->Kw : p->Lw;
  Staged<double> xs, ys;
  int rc = xs.in(x, (size_t)in_len * nvec, p->stream);
  if (rc) return rc;
  rc = ys.out(y, (size_t)out_len * nvec, p->stream);
  if (rc) return rc;
  void* scratch = p->scratch;
  void* tmp = nullptr;
  if (!p->small && nvec > 1) {
    CK(dev_alloc(&tmp, ((size_t)1 << p->g.lg_n) * sizeof(cplx<df64>) * nvec, p->stream));
    scratch = tmp;
  }
  launch_matvec_d(p->g, p->opts.precision, t, xs.dev, in_len, ys.dev, out_len, nvec, p->chat, scratch, p->stream);
  CHECK_LAUNCH();
  if (p->fexp) {  // products of the scaled series, back in the caller's units
    scale_copy(ys.dev, ys.dev, out_len * nvec, p->fexp, p->stream);
    CHECK_LAUNCH();
  }
  if (tmp) CK(cudaFreeAsync(tmp, p->stream));
  rc = ys.finish();
  if (rc) return rc;
  if (ys.needs_sync() || xs.owned) CK(cudaStreamSynchronize(p->stream));
  return SSA_OK;
}

// ------------------------------------------------------------------ Lanczos
static int ensure_workspace(ssa_plan_t p, int d) {
  Workspace& w = p->ws;
  if (w.dcap >= d) return SSA_OK;
  cudaStream_t st = p->stream;
  p->drop_cycles();  // their kernels point into the old workspace
  w.release(st);
  const int cols = d + 2;
  w.ldu = (p->Lw + 3) / 4 * 4;
  w.ldv = (p->Kw + 3) / 4 * 4;
  w.ldb = d + 2;
  const int64_t dimmax = p->Kw > p->Lw ? p->Kw : p->Lw;
  const int G = reorth_blocks(dimmax);
  for (int i = 0; i < 2; ++i) {
    CK(malloc_async(&w.Ub[i], (size_t)w.ldu * cols * sizeof(df64), st));
    CK(malloc_async(&w.Vb[i], (size_t)w.ldv * cols * sizeof(df64), st));
    CK(cudaMemsetAsync(w.Ub[i], 0, (size_t)w.ldu * cols * sizeof(df64), st));
    CK(cudaMemsetAsync(w.Vb[i], 0, (size_t)w.ldv * cols * sizeof(df64), st));
  }
  CK(malloc_async(&w.B, (size_t)w.ldb * w.ldb * sizeof(df64), st));
  CK(malloc_async(&w.y, (size_t)((dimmax + 3) / 4 * 4) * sizeof(df64), st));
  w.rw.ldp = MAXCOL + 1;
  CK(malloc_async(&w.rw.part, (size_t)G * w.rw.ldp * sizeof(df64), st));
  w.rw.ldp2 = FUSED_MAXCOL + 1;
  CK(malloc_async(&w.rw.part2, (size_t)fused_tiles(dimmax) * w.rw.ldp2 * sizeof(df64), st));
  reorth_setup();
  CK(malloc_async(&w.rw.coop, (size_t)coop_blocks() * (MAXCOL + 1) * sizeof(df64), st));
  CK(malloc_async(&w.rw.h, (MAXCOL + 1) * sizeof(df64), st));
  CK(malloc_async(&w.rw.h2, (MAXCOL + 1) * sizeof(df64), st));
  CK(malloc_async(&w.rw.gate, sizeof(int), st));
  CK(malloc_async(&w.rw.run, sizeof(int), st));
  CK(malloc_async(&w.rw.skip, sizeof(int), st));
  CK(malloc_async(&w.rw.nrm, sizeof(df64), st));
  CK(malloc_async(&w.rw.counter, sizeof(int), st));
  CK(cudaMemsetAsync(w.rw.counter, 0, sizeof(int), st));
  const size_t sq = (size_t)cols * cols * sizeof(df64);
  CK(malloc_async(&w.sw.A, sq, st));
  CK(malloc_async(&w.sw.W, sq, st));
  CK(malloc_async(&w.sw.P, sq, st));
  CK(malloc_async(&w.sw.Q, sq, st));
  CK(malloc_async(&w.sw.sigma, cols * sizeof(df64), st));
  CK(malloc_async(&w.sw.resid, cols * sizeof(double), st));
  CK(malloc_async(&w.sw.sigma_d, cols * sizeof(double), st));
  CK(malloc_async(&w.sw.conv, sizeof(int), st));
  if (p->opts.reorth == SSA_REORTH_NONE) {
    CK(malloc_async(&w.sw2.A, sq, st));
    CK(malloc_async(&w.sw2.W, sq, st));
    CK(malloc_async(&w.sw2.P, sq, st));
    CK(malloc_async(&w.sw2.Q, sq, st));
    CK(malloc_async(&w.sw2.sigma, cols * sizeof(df64), st));
    CK(malloc_async(&w.sw2.resid, cols * sizeof(double), st));
    CK(malloc_async(&w.sw2.sigma_d, cols * sizeof(double), st));
    CK(malloc_async(&w.sw2.conv, sizeof(int), st));
  }
  CK(malloc_async(&w.est, sizeof(df64), st));
  CK(malloc_async(&w.dummy, sizeof(df64), st));
  CK(malloc_async(&w.flag, sizeof(int), st));
  CK(malloc_async(&w.status, sizeof(unsigned), st));
  w.rw.status = w.status;
  CK(malloc_async(&w.sgn, cols * sizeof(int), st));
  w.pro.lde = cols;
  CK(malloc_async(&w.pro.M, (size_t)cols * cols * sizeof(float), st));
  CK(malloc_async(&w.pro.N, (size_t)cols * cols * sizeof(float), st));
  CK(malloc_async(&w.pro.force, 2 * sizeof(int), st));
  w.dcap = d;
  return SSA_OK;
}

static int refine_sigma(ssa_plan_t p, ssa_decomp_s* res, int k);

// The Cullum-Willoughby selection (host only): sigma (c values, descending) are the singular
// values of the projected matrix, sigma_hat (c_hat values) those of the matrix without its first
// row, resid the residual estimates of sigma's Ritz pairs.  Values agree within 1e-10 sigma_1;
// values at or below that are not candidates.  Walking sigma's groups of agreeing values in
// descending order, a group of one value that agrees with some sigma_hat value is spurious; any
// other group keeps its member with the smallest residual (lowest index on ties).  The first k kept
// indices, padded with the largest unused indices when fewer pass, are written to keep in
// ascending order; *converged = k passed and each kept residual is <= tol sigma_1.
static int cw_select(const double* sig, int c, const double* sig2, int c2, const double* res, int k, double tol,
                     int32_t* keep_out, int* converged) {
  if (c < 1 || k < 1 || k > c || c2 < 0) return SSA_EINVAL;
  const double same = 1e-10 * sig[0];  // two singular values agree within this
  std::vector<int> keep;
  for (int i = 0; i < c && (int)keep.size() < k && sig[i] > same;) {
    int j = i;
    while (j + 1 < c && sig[j + 1] >= sig[i] - same) ++j;
    bool spurious = false;
    if (j == i)
      for (int t = 0; t < c2; ++t)
        if (std::fabs(sig2[t] - sig[i]) <= same) spurious = true;
    if (!spurious) {  // of several copies, the one whose Ritz pair has the smallest residual
      int best = i;
      for (int t = i + 1; t <= j; ++t)
        if (res[t] < res[best]) best = t;
      keep.push_back(best);
    }
    i = j + 1;
  }
  bool ok = (int)keep.size() == k;
  for (int i : keep) ok = ok && res[i] <= tol * sig[0];
  std::vector<char> used(c, 0);
  for (int i : keep) used[i] = 1;
  for (int i = 0; i < c && (int)keep.size() < k; ++i)
    if (!used[i]) keep.push_back(i);
  std::sort(keep.begin(), keep.end());
  for (int m = 0; m < k; ++m) keep_out[m] = keep[m];
  *converged = ok ? 1 : 0;
  return SSA_OK;
}

extern "C" int ssa_cw_filter(const double* sigma, int c, const double* sigma_hat, int c_hat, const double* resid,
                             int k, double tol, int32_t* keep, int* converged) {
  REQ(sigma != nullptr && resid != nullptr && keep != nullptr && converged != nullptr &&
          (sigma_hat != nullptr || c_hat == 0),
      "NULL argument");
  REQ(c >= 1 && k >= 1 && k <= c && c_hat >= 0, "need 1 <= k <= c and c_hat >= 0");
  for (int i = 0; i < c; ++i) {
    REQ(std::isfinite(sigma[i]) && std::isfinite(resid[i]), "non-finite sigma or residual at %d", i);
    REQ(i == 0 || sigma[i] <= sigma[i - 1], "sigma must be in descending order");
  }
  return cw_select(sigma, c, sigma_hat, c_hat, resid, k, tol, keep, converged);
}

// Cullum-Willoughby filtering of a bidiagonalisation run without reorthogonalisation
// (section 3.2.1): the projected matrix B (r x c) is the Golub-Kahan tridiagonal of the
// Lanczos process started from u_1; a simple singular value of B that is also a singular
// value of B without its first row is spurious, and copies of a value count once (the copy
// with the smallest residual is kept).  The first k values that pass become the first k
// columns of the SVD outputs (P, Q, sigma, residuals), in descending order; when fewer than
// k pass, the largest remaining values fill the rest and the result is not converged.  converged: k values passed and each residual
// is <= tol sigma_1.
static int ghost_filter(Workspace& w, int r, int c, int k, double tol, int* converged, cudaStream_t s) {
  w.sw2.max_sweeps = w.sw.max_sweeps;
  w.sw2.rot_tol = w.sw.rot_tol;
  launch_small_svd(w.B + w.ldb, w.ldb, r - 1, c, w.sw2, 0, 1.0, w.est, w.status, s);
  CHECK_LAUNCH();
  std::vector<double> sig(c), sig2(c), res(c);
  CK(cudaMemcpyAsync(sig.data(), w.sw.sigma_d, c * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sig2.data(), w.sw2.sigma_d, c * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(res.data(), w.sw.resid, c * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int32_t> keep(k);
  int ok = 0;
  if (cw_select(sig.data(), c, sig2.data(), c, res.data(), k, tol, keep.data(), &ok) != SSA_OK) return SSA_EINVAL;
  *converged = ok;
  // gather the kept columns into the first k places (host round trip of the small matrices)
  std::vector<df64> P((size_t)r * c), Q((size_t)c * c), sg(c);
  std::vector<double> sd(c);
  CK(cudaMemcpyAsync(P.data(), w.sw.P, P.size() * sizeof(df64), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(Q.data(), w.sw.Q, Q.size() * sizeof(df64), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sg.data(), w.sw.sigma, c * sizeof(df64), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sd.data(), w.sw.sigma_d, c * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<df64> P2((size_t)r * k), Q2((size_t)c * k), sg2(k);
  std::vector<double> sd2(k), res2(k);
  for (int m = 0; m < k; ++m) {
    const int i = keep[m];
    std::copy(P.begin() + (size_t)i * r, P.begin() + (size_t)(i + 1) * r, P2.begin() + (size_t)m * r);
    std::copy(Q.begin() + (size_t)i * c, Q.begin() + (size_t)(i + 1) * c, Q2.begin() + (size_t)m * c);
    sg2[m] = sg[i];
    sd2[m] = sd[i];
    res2[m] = res[i];
  }
  CK(cudaMemcpyAsync(w.sw.P, P2.data(), P2.size() * sizeof(df64), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.sw.Q, Q2.data(), Q2.size() * sizeof(df64), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.sw.sigma, sg2.data(), k * sizeof(df64), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.sw.sigma_d, sd2.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.sw.resid, res2.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host vectors go out of scope
  return SSA_OK;
}

static int lanczos(ssa_plan_t p, int k, ssa_decomp_s* res) {
  const int prec = p->opts.precision;
  const int64_t Lw = p->Lw, Kw = p->Kw;
  const int64_t mn = Lw < Kw ? Lw : Kw;
  const bool none = prec != SSA_PREC_F32C && p->opts.reorth == SSA_REORTH_NONE;
  int d = p->opts.krylov_dim > 0 ? p->opts.krylov_dim : (2 * k > k + 32 ? 2 * k : k + 32);
  // without reorthogonalisation one cycle of four times the usual length (copies of the converged
  // triples take up part of it; three times left the last residuals near 2e-12 sigma_1 at
  // k = 12-16), within the largest basis
  if (none && p->opts.krylov_dim <= 0) d = 4 * d < MAXCOL - 2 ? 4 * d : MAXCOL - 2;
  if (d > mn) d = (int)mn;
  if (d < k) d = k;
  REQ(d <= MAXCOL - 2, "Krylov dimension %d exceeds %d", d, MAXCOL - 2);
  // keep k + ceil((d - k) / 5) Ritz pairs: fewer kept columns make the
  // reorthogonalisation of each cycle cheaper and cost few extra restarts
  int kk = p->opts.keep > 0 ? p->opts.keep : k + (d - k + 4) / 5;
  if (kk > d - 1) kk = d - 1;
  if (kk < k) kk = k;
  double tol = p->opts.tol;
  if (!(tol > 0)) tol = prec == SSA_PREC_F32C ? 1e-7 * std::sqrt((double)ilog2(p->g.M)) : 1e-12;
  int rc = ensure_workspace(p, d);
  if (rc) return rc;
  Workspace& w = p->ws;
  cudaStream_t s = p->stream;
  int cur = 0;
  df64* U = w.Ub[cur];
  df64* V = w.Vb[cur];
  CK(cudaMemsetAsync(w.flag, 0, sizeof(int), s));
  CK(cudaMemsetAsync(w.status, 0, sizeof(unsigned), s));
  w.sw.max_sweeps = 60;
  w.sw.rot_tol = 1e-13f;
  const uint64_t seed = p->opts.seed;
  // counter streams of the random vectors: 0 the starting vector, 1 its breakdown replacement, and
  // 2 + 2 j (+1 on the v side) the replacement of the j-th vector of a side, so that a half-step's
  // launches depend only on its position (a cycle replays from a CUDA graph unchanged)
  auto sid = [](int j, bool vside) { return (uint64_t)2 + 2 * (uint64_t)j + (vside ? 1 : 0); };
  int64_t matvecs = 0;
  // one reorthogonalisation pass suffices when the products are FP32 (their
  // error, ~1e-7 sigma_1, is far above one pass's df64 orthogonality)
  const int reorth = prec == SSA_PREC_F32C ? REORTH_ONCE : REORTH_GATED;
  // partial reorthogonalisation keeps sigma at working accuracy only while no thick restart
  // happens (the coefficients it leaves out, up to sqrt(eps) ||w||, would enter the restarted
  // arrow matrix): a first cycle that does not converge starts over with full Gram-Schmidt
  bool pro = prec != SSA_PREC_F32C && p->opts.reorth == SSA_REORTH_PRO;
  w.rw.skip_tau = prec == SSA_PREC_F32C || pro ? 0.0 : p->opts.reorth_skip;
  w.rw.grid_cap = p->opts.grid_cap;
  w.pro.eps = 1.4e-14f;  // relative error of the double-float products (2^-46)
  int r = 1, c = 0;
  auto side = [&](bool vside) -> int {
    // v-side: alpha v_{c+1} = X^T u_r - ... ; u-side: beta u_{r+1} = X v_c - ...
    df64* Qb = vside ? V : U;
    const int64_t ldq = vside ? w.ldv : w.ldu;
    const int64_t dim = vside ? Kw : Lw;
    const int ncols = vside ? c : r;
    const df64* src = vside ? U + (int64_t)(r - 1) * w.ldu : V + (int64_t)(c - 1) * w.ldv;
    df64* bentry = vside ? w.B + (int64_t)(r - 1) * w.ldb + c : w.B + (int64_t)r * w.ldb + (c - 1);
    launch_matvec_df(p->g, prec, vside ? 1 : 0, src, 0, w.y, 0, 1, p->chat, p->scratch, s);
    ++matvecs;
    int mode = reorth;
    if (none && ncols > 0) {
      // no reorthogonalisation (section 3.2.1): the recurrence's one coupling and ||w||^2
      CK((cudaError_t)launch_pro_pre(w.y, dim, vside ? V + (int64_t)(c - 1) * w.ldv : U + (int64_t)(r - 1) * w.ldu,
                                     w.B + (int64_t)(r - 1) * w.ldb + (c - 1), w.rw, w.pro, w.B, w.ldb,
                                     vside ? 1 : 0, ncols, vside ? r - 1 : c - 1, 0, 0, -1, w.est, s));
      w.rw.nrm_blocks = 0;  // the normalisation takes *rw.nrm
      w.rw.skip_flag = nullptr;
      df64* qcol = Qb + (int64_t)ncols * ldq;
      CK((cudaError_t)launch_normalize_coop(w.y, dim, w.rw, qcol, bentry, w.est, Qb, ldq, ncols, seed,
                                            sid(ncols, vside), w.status, s));
      CHECK_LAUNCH();
      if (vside) ++c;
      else ++r;
      return SSA_OK;
    }
    if (pro && ncols > 0) {
      // partial reorthogonalisation (first cycle only): subtract the one known coupling B[r-1][c-1]
      // (to v_{c-1} on the v side, to u_{r-1} on the u side), update the estimates and decide on
      // the device whether the Gram-Schmidt passes run
      const df64* coef = w.B + (int64_t)(r - 1) * w.ldb + (c - 1);
      const df64* qprev = vside ? V + (int64_t)(c - 1) * w.ldv : U + (int64_t)(r - 1) * w.ldu;
      CK((cudaError_t)launch_pro_pre(w.y, dim, qprev, coef, w.rw, w.pro, w.B, w.ldb, vside ? 1 : 0, ncols,
                                     vside ? r - 1 : c - 1, ncols, vside ? r : c, vside ? c - 1 : r - 1, w.est, s));
      mode = REORTH_PRO;
    }
    launch_cgs2(Qb, ldq, ncols, w.y, dim, w.rw, mode, s);
    df64* qcol = Qb + (int64_t)ncols * ldq;
    CK((cudaError_t)launch_normalize_coop(w.y, dim, w.rw, qcol, bentry, w.est, Qb, ldq, ncols, seed,
                                          sid(ncols, vside), w.status, s));
    CHECK_LAUNCH();
    if (vside) ++c;
    else ++r;
    return SSA_OK;
  };
  // p_0 (Algorithm 1): seeded uniform(-1, 1) from counter stream 0, normalised into u_1; then v_1
  auto start = [&]() -> int {
    CK(cudaMemsetAsync(w.B, 0, (size_t)w.ldb * w.ldb * sizeof(df64), s));
    CK(cudaMemsetAsync(w.est, 0, sizeof(df64), s));
    if (pro || none) launch_pro_reset(w.pro, s);
    launch_random_fill(w.y, Lw, seed, 0, s);
    launch_cgs2(U, w.ldu, 0, w.y, Lw, w.rw, reorth, s);
    CK((cudaError_t)launch_normalize_coop(w.y, Lw, w.rw, U, w.dummy, w.est, U, w.ldu, 0, seed, 1,
                                          w.status, s));
    CHECK_LAUNCH();
    r = 1;
    c = 0;
    return side(true);
  };
  // one cycle of half-steps up to the Krylov dimension; every decision inside it is taken on the
  // device, so its launches depend only on (cur, r, c, d, mode) and it replays from a CUDA graph
  auto plain_cycle = [&]() -> int {
    while (c < d + 1) {
      int e = side(false);
      if (e) return e;
      e = side(true);
      if (e) return e;
    }
    return SSA_OK;
  };
  const int64_t call = ++p->lanczos_calls;
  auto run_cycle = [&]() -> int {
    if (prof_enabled()) return plain_cycle();  // per-launch events and host reads: no graph
    int idx = -1;
    for (size_t i = 0; i < p->cycles.size(); ++i) {
      const auto& e = p->cycles[i];
      if (e.cur == cur && e.r0 == r && e.c0 == c && e.d == d && e.pro == pro && e.none == none) idx = (int)i;
    }
    if (idx < 0) {  // first time: run it and remember the shape
      p->cycles.push_back({cur, r, c, d, pro, none, call, false, false, nullptr, 0, 0, 0, 0});
      return plain_cycle();
    }
    if (p->cycles[idx].failed || p->cycles[idx].first_call == call) return plain_cycle();
    if (p->cycles[idx].captured) {
      auto& e = p->cycles[idx];
      CK(cudaGraphLaunch(e.exec, s));
      prof_add_launches(e.launches);
      r += e.dr;
      c += e.dc;
      matvecs += e.dmv;
      return SSA_OK;
    }
    // second time: capture (nothing runs during the capture), instantiate, launch
    const int r0 = r, c0 = c;
    const int64_t mv0 = matvecs;
    const uint64_t l0 = prof_thread_launches();
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    int rc2 = e == cudaSuccess ? plain_cycle() : SSA_ECUDA;
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(s, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc2 == SSA_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    const uint64_t nl = prof_thread_launches() - l0;
    const int dr = r - r0, dc = c - c0;
    const int64_t dmv = matvecs - mv0;
    // the captured launches did not run: undo the host-side bookkeeping
    r = r0;
    c = c0;
    matvecs = mv0;
    prof_sub_launches(nl);
    if (rc2 != SSA_OK || e != cudaSuccess || !exec) {  // not capturable here: run it as before
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      p->cycles[idx].failed = true;
      return plain_cycle();
    }
    auto& ent = p->cycles[idx];
    ent.exec = exec;
    ent.captured = true;
    ent.launches = nl;
    ent.dr = dr;
    ent.dc = dc;
    ent.dmv = dmv;
    CK(cudaGraphLaunch(exec, s));
    prof_add_launches(nl);
    r += ent.dr;
    c += ent.dc;
    matvecs += ent.dmv;
    return SSA_OK;
  };
  int restarts = 0, converged = 0;
  rc = start();
  if (rc) return rc;
  unsigned status = 0;
  for (;;) {
    rc = run_cycle();
    if (rc) return rc;
    const int cp = c - 1;
    launch_small_svd(w.B, w.ldb, r, cp, w.sw, k, tol, w.est, w.status, s);
    CHECK_LAUNCH();
    CK(cudaMemcpyAsync(&converged, w.sw.conv, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&status, w.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    unsigned sfault = 0;
    CK((cudaError_t)spectral_fault_read(&sfault, s));
    CK(cudaStreamSynchronize(s));
    if (sfault) {
      set_err("a bounded wait for a bulk copy into shared memory ran out in the FFT products");
      return SSA_ECUDA;
    }
    if (prof_enabled()) prof_flush();
    if (status & SSA_DEV_NONFINITE) {
      set_err("non-finite value in the Lanczos recurrence");
      return SSA_ENUMERIC;
    }
    if (none) {  // one cycle, then the Cullum-Willoughby filter picks the k triples
      rc = ghost_filter(w, r, cp, k, tol, &converged, s);
      if (rc) return rc;
      break;
    }
    if (converged || restarts >= p->opts.max_restarts || kk >= cp) break;
    if (pro) {  // the first cycle did not converge: start over with full Gram-Schmidt
      pro = false;
      ++restarts;
      rc = start();
      if (rc) return rc;
      continue;
    }
    // thick restart: U <- U P[:, :kk], V <- [V Q[:, :kk], v_{c}], B <- [diag | rho]
    const int nxt = cur ^ 1;
    launch_ritz(U, w.ldu, r, w.sw.P, r, kk, w.Ub[nxt], w.ldu, Lw, s);
    launch_ritz(V, w.ldv, cp, w.sw.Q, cp, kk, w.Vb[nxt], w.ldv, Kw, s);
    launch_copy_df(V + (int64_t)cp * w.ldv, w.Vb[nxt] + (int64_t)kk * w.ldv, Kw, s);
    launch_restart_B(w.B, w.ldb, w.ldb, w.sw, r, kk, cp, s);
    CHECK_LAUNCH();
    cur = nxt;
    U = w.Ub[cur];
    V = w.Vb[cur];
    r = kk;
    c = kk + 1;
    ++restarts;
  }
  // Ritz vectors for the k wanted triples
  const int nxt = cur ^ 1;
  df64* Uf = w.Ub[nxt];
  df64* Vf = w.Vb[nxt];
  const int cp = c - 1;
  launch_ritz(U, w.ldu, r, w.sw.P, r, k, Uf, w.ldu, Lw, s);
  launch_ritz(V, w.ldv, cp, w.sw.Q, cp, k, Vf, w.ldv, Kw, s);
  if (none) {  // the bases are not orthonormal: unit Ritz vectors
    launch_normalize_cols(Uf, w.ldu, Lw, k, s);
    launch_normalize_cols(Vf, w.ldv, Kw, k, s);
  }
  CHECK_LAUNCH();
  // sign rule on the user's left vectors
  const df64* Uuser = p->transposed ? Vf : Uf;
  const int64_t lduser = p->transposed ? w.ldv : w.ldu;
  const int64_t Luser = p->transposed ? Kw : Lw;
  launch_sign(Uuser, lduser, Luser, k, w.sgn, s);
  launch_store_cols(Uf, w.ldu, Lw, k, w.sgn, p->transposed ? res->V : res->U, Lw, s);
  launch_store_cols(Vf, w.ldv, Kw, k, w.sgn, p->transposed ? res->U : res->V, Kw, s);
  // working-orientation copies for Hankelization
  CK(cudaMemcpy2DAsync(res->Uw, Lw * sizeof(df64), Uf, w.ldu * sizeof(df64), Lw * sizeof(df64), k,
                       cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpy2DAsync(res->Vw, Kw * sizeof(df64), Vf, w.ldv * sizeof(df64), Kw * sizeof(df64), k,
                       cudaMemcpyDeviceToDevice, s));
  scale_copy(w.sw.sigma_d, res->sigma, k, p->fexp, s);  // back to the caller's units
  scale_copy(w.sw.resid, res->resid, k, p->fexp, s);
  CHECK_LAUNCH();
  CK(cudaStreamSynchronize(s));
  res->k = k;
  res->d = d;
  res->converged = converged;
  res->restarts = restarts;
  if (p->opts.refine == SSA_REFINE_ON) {
    rc = refine_sigma(p, res, k);
    if (rc) return rc;
    matvecs += k;
  }
  res->matvecs = matvecs;
  // Uw / Vw keep the unsigned vectors: Hankelizing sigma u v^T does not
  // depend on flipping u and v together.
  return converged ? SSA_OK : SSA_ENOCONV;
}

// Native-FP64 tables and spectrum of the plan's series (the four-step order
// is kept unless the native product runs in one CTA).
static int native_spectrum(ssa_plan_t p, Geom& g64) {
  Geom& g = p->g;
  const int64_t P = (int64_t)1 << g.lg_P;
  const int64_t M = g.M;
  const int64_t nA = M >> g.tws, nB = (int64_t)1 << g.tws;
  const int64_t n = (int64_t)1 << g.lg_n;
  if (!p->tw64) {
    std::vector<cplx<double>> htw(P), hA(nA), hB(nB);
    for (int64_t m = 0; m < P; ++m) htw[m] = tw_entry64(m, P);
    for (int64_t m = 0; m < nA; ++m) hA[m] = tw_entry64(m << g.tws, M);
    for (int64_t m = 0; m < nB; ++m) hB[m] = tw_entry64(m, M);
    CK(malloc_async(&p->tw64, P * sizeof(cplx<double>), p->stream));
    CK(malloc_async(&p->tA64, nA * sizeof(cplx<double>), p->stream));
    CK(malloc_async(&p->tB64, nB * sizeof(cplx<double>), p->stream));
    CK(malloc_async(&p->chat64, (n + 1) * sizeof(cplx<double>), p->stream));
    CK(cudaMemcpyAsync(p->tw64, htw.data(), P * sizeof(cplx<double>), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->tA64, hA.data(), nA * sizeof(cplx<double>), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->tB64, hB.data(), nB * sizeof(cplx<double>), cudaMemcpyHostToDevice, p->stream));
  }
  g64 = g;
  g64.tw64 = p->tw64;
  g64.tA64 = p->tA64;
  g64.tB64 = p->tB64;
  const float scale = 1.0f / (4.0f * (float)n);
  launch_spectrum64(g64, p->f_dev, p->chat64, native_small(g64) ? 1 : 0, scale, p->scratch, p->stream);
  CHECK_LAUNCH();
  return SSA_OK;
}

// sigma_i <- u_i^T (X v_i) with native-FP64 products, in chunks of vectors
// (the four-step product needs n complex doubles of scratch per vector).
// Returned triples are re-sorted if two nearly equal values swapped.
static int refine_sigma(ssa_plan_t p, ssa_decomp_s* res, int k) {
  Geom g64{};
  int rc = native_spectrum(p, g64);
  if (rc) return rc;
  cudaStream_t s = p->stream;
  const int64_t Lw = p->Lw, Kw = p->Kw;
  const double* Ui = p->transposed ? res->V : res->U;  // working orientation, columns signed alike
  const double* Vi = p->transposed ? res->U : res->V;
  const int64_t n = (int64_t)1 << g64.lg_n;
  const bool small = native_small(g64);
  int chunk = small ? k : (int)std::max<int64_t>(1, std::min<int64_t>(k, ((int64_t)256 << 20) / (n * 16)));
  double* Y = nullptr;
  void* scr = nullptr;
  CK(dev_alloc(&Y, (size_t)Lw * chunk * sizeof(double), s));
  if (!small && chunk > 1) CK(dev_alloc(&scr, (size_t)n * chunk * sizeof(cplx<double>), s));
  for (int c0 = 0; c0 < k; c0 += chunk) {
    const int nb = std::min(chunk, k - c0);
    launch_matvec_native(g64, 0, Vi + (int64_t)c0 * Kw, Kw, Y, Lw, nb, p->chat64, scr ? scr : p->scratch, s);
    launch_col_dots(Ui + (int64_t)c0 * Lw, Lw, Y, Lw, Lw, nb, res->sigma + c0, s);
  }
  scale_copy(res->sigma, res->sigma, k, p->fexp, s);  // products of the scaled series
  CHECK_LAUNCH();
  if (scr) CK(cudaFreeAsync(scr, s));
  CK(cudaFreeAsync(Y, s));
  std::vector<double> sg(k);
  CK(cudaMemcpyAsync(sg.data(), res->sigma, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool sorted = true;
  for (int i = 1; i < k; ++i) sorted = sorted && sg[i - 1] >= sg[i];
  if (sorted) return SSA_OK;
  std::vector<int> perm(k);
  for (int i = 0; i < k; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return sg[a] > sg[b]; });
  auto permute = [&](void* base, size_t colbytes) -> int {
    void* tmp = nullptr;
    CK(dev_alloc(&tmp, colbytes * k, s));
    CK(cudaMemcpyAsync(tmp, base, colbytes * k, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < k; ++i)
      if (perm[i] != i)
        CK(cudaMemcpyAsync(static_cast<char*>(base) + colbytes * i, static_cast<char*>(tmp) + colbytes * perm[i],
                           colbytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaFreeAsync(tmp, s));
    return SSA_OK;
  };
  if ((rc = permute(res->sigma, sizeof(double)))) return rc;
  if ((rc = permute(res->resid, sizeof(double)))) return rc;
  if ((rc = permute(res->U, p->L * sizeof(double)))) return rc;
  if ((rc = permute(res->V, p->K * sizeof(double)))) return rc;
  if ((rc = permute(res->Uw, Lw * sizeof(df64)))) return rc;
  if ((rc = permute(res->Vw, Kw * sizeof(df64)))) return rc;
  CK(cudaStreamSynchronize(s));
  return SSA_OK;
}

namespace ssa {
int64_t plan_path_bytes(int64_t N, int64_t L, int k, int precision) {
  const int64_t K = N - L + 1;
  const int64_t Lw = L < K ? L : K, Kw = L < K ? K : L;
  int64_t d = std::max<int64_t>(2 * k, k + 32);
  d = std::min(d, Lw);
  d = std::max<int64_t>(d, k);
  const int64_t cols = d + 2;
  int64_t M = 4;
  while (M < N) M *= 2;
  const int64_t n = M / 2;
  const int64_t ldu = (Lw + 3) / 4 * 4, ldv = (Kw + 3) / 4 * 4;
  int64_t b = 0;
  b += 2 * (ldu + ldv) * cols * 8;                                       // two basis pairs
  b += cols * cols * 8 * 5 + ((Kw + 3) / 4 * 4) * 8;                     // B, SVD work, y
  b += (int64_t)reorth_blocks(Kw) * (MAXCOL + 1) * 8;                    // partial sums
  b += (int64_t)fused_tiles(Kw) * (FUSED_MAXCOL + 1) * 8;
  b += (int64_t)coop_blocks() * (MAXCOL + 1) * 8;
  b += (2 * n + 3 * (n + 1)) * 16 + N * 8;                               // tables, spectrum, scratch, f
  b += (L + K) * k * 16 + k * 16;                                        // results (double and df64)
  (void)precision;
  return b + (4 << 20);                                                  // allocator granularity
}
}  // namespace ssa

extern "C" void ssa_decomp_destroy(ssa_decomp_t d) {
  if (!d) return;
  cudaStream_t st = d->plan ? d->plan->stream : nullptr;
  free_async(d->sigma, st);
  free_async(d->resid, st);
  free_async(d->U, st);
  free_async(d->V, st);
  free_async(d->Uw, st);
  free_async(d->Vw, st);
  delete d;
}

extern "C" int ssa_decompose(ssa_plan_t p, const double* f, int k, ssa_decomp_t* out) {
  REQ(p != nullptr && out != nullptr, "NULL argument");
  *out = nullptr;
  const int64_t mn = p->Lw;
  REQ(k >= 1 && k <= mn, "need 1 <= k <= min(L, K) = %lld (got %d)", (long long)mn, k);
  if (f) {
    int rc = set_series(p, f);
    if (rc) return rc;
  }
  REQ(p->has_series, "no series given");
  ssa_decomp_s* d = new (std::nothrow) ssa_decomp_s();
  if (!d) return SSA_ENOMEM;
  d->plan = p;
#define DK(x)                                       \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) {                        \
      set_err("%s: %s", #x, cudaGetErrorString(e_)); \
      ssa_decomp_destroy(d);                        \
      return e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA; \
    }                                               \
  } while (0)
  DK(malloc_async(&d->sigma, k * sizeof(double), p->stream));
  DK(malloc_async(&d->resid, k * sizeof(double), p->stream));
  DK(malloc_async(&d->U, (size_t)p->L * k * sizeof(double), p->stream));
  DK(malloc_async(&d->V, (size_t)p->K * k * sizeof(double), p->stream));
  DK(malloc_async(&d->Uw, (size_t)p->Lw * k * sizeof(df64), p->stream));
  DK(malloc_async(&d->Vw, (size_t)p->Kw * k * sizeof(df64), p->stream));
#undef DK
  int rc = lanczos(p, k, d);
  if (rc != SSA_OK && rc != SSA_ENOCONV) {
    ssa_decomp_destroy(d);
    return rc;
  }
  *out = d;
  return rc;
}

extern "C" int ssa_decomp_info(ssa_decomp_t d, int* k, int* converged, int* restarts, int64_t* matvecs,
                               int* krylov_dim) {
  REQ(d != nullptr, "decomposition is NULL");
  if (k) *k = d->k;
  if (converged) *converged = d->converged;
  if (restarts) *restarts = d->restarts;
  if (matvecs) *matvecs = d->matvecs;
  if (krylov_dim) *krylov_dim = d->d;
  return SSA_OK;
}

extern "C" int ssa_decomp_get(ssa_decomp_t d, double* sigma, double* U, double* V, double* resid) {
  REQ(d != nullptr, "decomposition is NULL");
  const ssa_plan_t p = d->plan;
  cudaStream_t s = p->stream;
  if (sigma) CK(cudaMemcpyAsync(sigma, d->sigma, d->k * sizeof(double), cudaMemcpyDefault, s));
  if (resid) CK(cudaMemcpyAsync(resid, d->resid, d->k * sizeof(double), cudaMemcpyDefault, s));
  if (U) CK(cudaMemcpyAsync(U, d->U, (size_t)p->L * d->k * sizeof(double), cudaMemcpyDefault, s));
  if (V) CK(cudaMemcpyAsync(V, d->V, (size_t)p->K * d->k * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return SSA_OK;
}

// validate CSR groups (host copies); indices in [0, r), disjoint
static int check_groups(const int32_t* off, const int32_t* idx, int m, int r, std::vector<int32_t>& hoff,
                        std::vector<int32_t>& hidx) {
  REQ(m >= 1, "need m >= 1 groups");
  REQ(off != nullptr && idx != nullptr, "NULL group arrays");
  hoff.resize(m + 1);
  if (is_device_ptr(off)) CK(cudaMemcpy(hoff.data(), off, (m + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  else std::memcpy(hoff.data(), off, (m + 1) * sizeof(int32_t));
  REQ(hoff[0] == 0, "grp_off[0] must be 0");
  for (int g = 0; g < m; ++g) REQ(hoff[g + 1] >= hoff[g], "grp_off must be non-decreasing");
  const int nidx = hoff[m];
  hidx.resize(nidx > 0 ? nidx : 1);
  if (nidx > 0) {
    if (is_device_ptr(idx)) CK(cudaMemcpy(hidx.data(), idx, nidx * sizeof(int32_t), cudaMemcpyDeviceToHost));
    else std::memcpy(hidx.data(), idx, nidx * sizeof(int32_t));
  }
  std::vector<char> seen(r, 0);
  for (int i = 0; i < nidx; ++i) {
    REQ(hidx[i] >= 0 && hidx[i] < r, "group index %d out of range [0, %d)", hidx[i], r);
    REQ(!seen[hidx[i]], "index %d appears in two groups", hidx[i]);
    seen[hidx[i]] = 1;
  }
  return SSA_OK;
}

static int hankel_common(ssa_plan_t p, const double* sigma_dev, const df64* Uw, int64_t ldu, const df64* Vw,
                         int64_t ldv, int r, const int32_t* grp_off, const int32_t* grp_idx, int m, double* out) {
  std::vector<int32_t> hoff, hidx;
  int rc = check_groups(grp_off, grp_idx, m, r, hoff, hidx);
  if (rc) return rc;
  cudaStream_t s = p->stream;
  int32_t *doff = nullptr, *didx = nullptr;
  CK(dev_alloc(&doff, (m + 1) * sizeof(int32_t), s));
  CK(dev_alloc(&didx, hidx.size() * sizeof(int32_t), s));
  CK(cudaMemcpyAsync(doff, hoff.data(), (m + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(didx, hidx.data(), hidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  Staged<double> os;
  rc = os.out(out, (size_t)m * p->N, s);
  if (rc) return rc;
  // sigma enters the double-float kernels scaled by 2^-e (max sigma in [1/2, 1)) and the result
  // is scaled back by 2^e: exact, and independent of the units of the series
  std::vector<double> hs(r);
  CK(cudaMemcpyAsync(hs.data(), sigma_dev, r * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double smax = 0.0;
  for (int i = 0; i < r; ++i) {
    REQ(std::isfinite(hs[i]), "sigma[%d] is not finite", i);
    smax = std::max(smax, std::fabs(hs[i]));
  }
  int e = 0;
  if (smax > 0.0) std::frexp(smax, &e);
  double* sig_scaled = nullptr;
  if (e != 0) {
    CK(dev_alloc(&sig_scaled, r * sizeof(double), s));
    scale_copy(sigma_dev, sig_scaled, r, -e, s);
  }
  // four-step sizes: scratch for as many groups per launch as fit in 2 GiB, and the per-round index lists
  const size_t per = hankel_scratch_bytes(p->g, p->opts.precision, 1);
  int rows = 1;
  void* hscr = nullptr;
  int* hidx_dev = nullptr;
  if (per > 0) {
    rows = (int)std::max<size_t>(1, std::min<size_t>((size_t)m, ((size_t)2 << 30) / per));
    CK(dev_alloc(&hscr, hankel_scratch_bytes(p->g, p->opts.precision, rows), s));
    CK(dev_alloc(&hidx_dev, 2 * std::max<size_t>(1, hidx.size()) * sizeof(int), s));
  }
  launch_hankel(p->g, p->opts.precision, Uw, ldu, Vw, ldv, sig_scaled ? sig_scaled : sigma_dev, doff, didx,
                hoff.data(), hidx.data(), m, os.dev, p->N, hscr, rows, hidx_dev, std::ldexp(1.0, e), s);
  CHECK_LAUNCH();
  if (hscr) CK(cudaFreeAsync(hscr, s));
  if (hidx_dev) CK(cudaFreeAsync(hidx_dev, s));
  if (sig_scaled) CK(cudaFreeAsync(sig_scaled, s));
  rc = os.finish();
  if (rc) return rc;
  CK(cudaFreeAsync(doff, s));
  CK(cudaFreeAsync(didx, s));
  // host group arrays must outlive the enqueue of the large-M path (done) and
  // the copies above; synchronise so hoff/hidx can be released safely
  CK(cudaStreamSynchronize(s));
  return SSA_OK;
}

extern "C" int ssa_reconstruct(ssa_decomp_t d, const int32_t* grp_off, const int32_t* grp_idx, int m, double* out) {
  REQ(d != nullptr && out != nullptr, "NULL argument");
  ssa_plan_t p = d->plan;
  return hankel_common(p, d->sigma, d->Uw, p->Lw, d->Vw, p->Kw, d->k, grp_off, grp_idx, m, out);
}

extern "C" int ssa_hankelize(ssa_plan_t p, const double* sigma, const double* U, int64_t ldu, const double* V,
                             int64_t ldv, int r, const int32_t* grp_off, const int32_t* grp_idx, int m, double* out) {
  REQ(p != nullptr && sigma != nullptr && U != nullptr && V != nullptr && out != nullptr, "NULL argument");
  REQ(r >= 1, "need r >= 1");
  REQ(ldu >= p->L && ldv >= p->K, "leading dimensions too small");
  cudaStream_t s = p->stream;
  Staged<double> ss, us, vs;
  int rc = ss.in(sigma, r, s);
  if (rc) return rc;
  rc = us.in(U, (size_t)ldu * (r - 1) + p->L, s);
  if (rc) return rc;
  rc = vs.in(V, (size_t)ldv * (r - 1) + p->K, s);
  if (rc) return rc;
  df64 *Uw = nullptr, *Vw = nullptr;
  CK(dev_alloc(&Uw, (size_t)p->Lw * r * sizeof(df64), s));
  CK(dev_alloc(&Vw, (size_t)p->Kw * r * sizeof(df64), s));
  // working orientation: X^T's left vectors are the user's V when L > K
  const double* uw_src = p->transposed ? vs.dev : us.dev;
  const double* vw_src = p->transposed ? us.dev : vs.dev;
  launch_double_to_df(uw_src, p->transposed ? ldv : ldu, Uw, p->Lw, p->Lw, r, s);
  launch_double_to_df(vw_src, p->transposed ? ldu : ldv, Vw, p->Kw, p->Kw, r, s);
  CHECK_LAUNCH();
  rc = hankel_common(p, ss.dev, Uw, p->Lw, Vw, p->Kw, r, grp_off, grp_idx, m, out);
  cudaFreeAsync(Uw, s);
  cudaFreeAsync(Vw, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return SSA_OK;
}
