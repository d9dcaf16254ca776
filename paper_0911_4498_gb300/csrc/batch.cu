// Batched decompositions: many independent series of uneven length in one
// persistent launch.  Each CTA takes series from a device work queue (largest
// first) and runs the whole method for one series at a time, in the CTA:
//   spectrum of the series (Algorithm 2 steps 1-2, double-float),
//   Golub-Kahan-Lanczos bidiagonalisation (Algorithm 1) with every product by
//   Algorithms 2/3 as a single-CTA FFT in shared memory, CGS2
//   reorthogonalisation (section 3.2.2) streaming the basis through shared
//   memory, thick restart (section 3.3) with the one-CTA Jacobi SVD of the
//   projected matrix, Ritz vectors and the sign rule.
// Per-CTA scratch (bases, projected matrix, SVD work, spectrum) lives in one
// slot of a pool sized for the largest series of the batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ssa.h"
#include "budget.h"
#include "fft.cuh"
#include "lanczos_dev.cuh"
#include "prof.h"
#include "spectral.h"

namespace ssa {

constexpr int BT = 512;                 // threads per CTA
constexpr int B_SMEM = 128 * 1024;      // dynamic shared memory (FFT buffer, reused by every phase)
constexpr int B_MAXD = 72;              // largest Krylov dimension of a batched series
constexpr int B_MAXC = B_MAXD + 2;      // basis columns / projected-matrix size
constexpr int B_FR = 64;                // CGS tile rows (32 lanes x 2 rows)
constexpr int B_NST = 3;                // CGS pipeline stages: 3 x 74 columns x 64 rows df64 (111 KB) and the
                                        // row partials fit the 128 KB buffer

struct BSeries {
  int64_t f_off, N, L, K;  // user sizes
  int64_t Lw, Kw;          // working orientation (Lw <= Kw)
  int transposed;
  int k, d, kk;
  int lg_n;                // n = M / 2
  int64_t out_u, out_v, out_s;
};

struct BCtx {
  const BSeries* ser;
  int nseries;
  const int* order;
  int* next;
  const double* f;
  double *out_U, *out_V, *out_sigma, *out_resid;
  int* out_info;  // per series: converged, restarts, matvecs, status
  const cplx<df64>* tw;
  int lg_P;
  const cplx<df64>* tA;
  const cplx<df64>* tB;
  int tws;
  int lg_Mmax;
  char* slots;
  int64_t slot_bytes;
  int64_t ldu, ldv;  // basis leading dimensions of a slot
  int nmax;          // largest n of the batch
  int precision;
  double tol;
  double skip_tau;  // skip level of the gated reorthogonalisation (0: no skip test)
  int max_restarts;
  uint64_t seed;
};

struct Slot {  // carved out of the CTA's slot
  df64 *U[2], *V[2], *B, *A, *W, *P, *Q, *T, *sigma, *y;
  cplx<df64>* chat;
  cplx<df64>* fscr;
  double *resid, *sigma_d;
};

SSA_D Slot carve(const BCtx& cx, int slot_id) {
  char* base = cx.slots + (int64_t)slot_id * cx.slot_bytes;
  Slot s;
  df64* p = reinterpret_cast<df64*>(base);
  for (int i = 0; i < 2; ++i) { s.U[i] = p; p += cx.ldu * B_MAXC; }
  for (int i = 0; i < 2; ++i) { s.V[i] = p; p += cx.ldv * B_MAXC; }
  s.B = p; p += B_MAXC * B_MAXC;
  s.A = p; p += B_MAXC * B_MAXC;
  s.W = p; p += B_MAXC * B_MAXC;
  s.P = p; p += B_MAXC * B_MAXC;
  s.Q = p; p += B_MAXC * B_MAXC;
  s.T = p; p += B_MAXC * B_MAXC;
  s.sigma = p; p += B_MAXC + 2;
  s.y = p; p += cx.ldv;
  s.chat = reinterpret_cast<cplx<df64>*>(p);
  s.fscr = s.chat + (cx.nmax + 2);
  double* d = reinterpret_cast<double*>(s.fscr + cx.nmax);
  s.resid = d;
  s.sigma_d = d + B_MAXC + 2;
  return s;
}

int64_t slot_bytes_for(int64_t ldu, int64_t ldv, int nmax) {
  int64_t dfs = 2 * ldu * B_MAXC + 2 * ldv * B_MAXC + 6 * B_MAXC * B_MAXC + (B_MAXC + 2) + ldv;
  int64_t bytes = dfs * 8 + (int64_t)(2 * nmax + 2) * 16 + 2 * (B_MAXC + 2) * 8;
  return (bytes + 255) / 256 * 256;
}

static int b_krylov_dim(int64_t Lw, int k) {
  int d = std::max(2 * k, k + 32);
  if (d > Lw) d = (int)Lw;
  if (d < k) d = k;
  return d;
}

bool batch_eligible(int64_t N, int64_t L, int k, int precision) {
  const int64_t K = N - L + 1;
  const int64_t Lw = L < K ? L : K;
  const int64_t nmax = precision == SSA_PREC_F32C ? 32768 : 16384;
  return N > 2 && N <= nmax && L > 1 && L < N && k >= 1 && k <= Lw && b_krylov_dim(Lw, k) <= B_MAXD;
}

int64_t batch_path_bytes(const std::vector<BatchItem>& items, int refine) {
  int64_t ldu = 4, ldv = 4, tot = 0, Mmax = 4;
  int nmax = 2;
  for (const BatchItem& it : items) {
    const int64_t K = it.N - it.L + 1;
    const int64_t Lw = it.L < K ? it.L : K, Kw = it.L < K ? K : it.L;
    int64_t M = 4;
    while (M < it.N) M *= 2;
    Mmax = std::max(Mmax, M);
    nmax = std::max(nmax, (int)(M / 2));
    ldu = std::max(ldu, (Lw + 3) / 4 * 4);
    ldv = std::max(ldv, (Kw + 3) / 4 * 4);
    tot += (it.L + K) * it.k * 8 + it.k * 16 + it.N * 8 + (int64_t)sizeof(BSeries) + 24;
  }
  static const int sms = [] {  // thread-safe one-time initialisation
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
  }();
  const int64_t nslots = std::min<int64_t>(sms, (int64_t)items.size());
  tot += nslots * slot_bytes_for(ldu, ldv, nmax);
  tot += (Mmax / 2 + 2 * Mmax) * 16 * (refine ? 2 : 1);  // twiddle tables
  return tot + (2 << 20);
}

// ---------------------------------------------------------------- spectrum
// c-hat = rFFT_M(c) in df64, scaled by 1/(4n), natural order.  n <= 8192 in
// shared memory; n = 16384 as two half-length FFTs (even / odd packed
// samples) combined through global scratch.
SSA_D double circ(const Geom& g, const double* f, int64_t j) {
  if (j < g.L) return f[g.N - g.L + j];
  const int64_t j0 = g.L + (g.M - g.N);
  return j >= j0 ? f[j - j0] : 0.0;
}

// Exponent e with max |f| = m 2^e, m in [1/2, 1) (0 for a zero series), the
// same in every thread.  The series enters the double-float spectrum scaled
// by 2^-e (exact), far from FP32's overflow and underflow whatever its
// units; sigma and the residuals are scaled back by 2^e at the end.
SSA_D int cta_series_exp(const double* f, int64_t n) {
  __shared__ double wm[BT / 32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += BT) m = fmax(m, fabs(f[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  m = wm[0];
  for (int i = 1; i < BT / 32; ++i) m = fmax(m, wm[i]);
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

SSA_D void cta_spectrum(const Geom& g, const double* f, double fs, cplx<df64>* chat, cplx<df64>* scr,
                        cplx<df64>* buf) {
  const int n = 1 << g.lg_n;
  const float s = 0.5f / (4.0f * (float)n);
  const cplx<df64>* Z;
  if (n <= 8192) {
    for (int t = threadIdx.x; t < n; t += BT)
      buf[t] = mk(df_from_double(fs * circ(g, f, 2 * (int64_t)t)),
                  df_from_double(fs * circ(g, f, 2 * (int64_t)t + 1)));
    __syncthreads();
    cta_fft<df64, BT, 8192, false>(buf, g.lg_n, 1, g.tw, g.lg_P);
    Z = buf;
  } else {
    const int h = n / 2;
    for (int par = 0; par < 2; ++par) {
      for (int t = threadIdx.x; t < h; t += BT) {
        const int64_t j = 4 * (int64_t)t + 2 * par;  // z[2t + par] = c[2(2t+par)] + i c[2(2t+par)+1]
        buf[t] = mk(df_from_double(fs * circ(g, f, j)), df_from_double(fs * circ(g, f, j + 1)));
      }
      __syncthreads();
      cta_fft<df64, BT, 8192, false>(buf, g.lg_n - 1, 1, g.tw, g.lg_P);
      if (par == 0) {
        for (int t = threadIdx.x; t < h; t += BT) scr[t] = buf[t];
        __syncthreads();
      }
    }
    for (int k = threadIdx.x; k < h; k += BT) {  // Z[k] = E[k] + W_n^k O[k], Z[k+h] = E[k] - W_n^k O[k]
      const cplx<df64> e = scr[k];
      const cplx<df64> t = c_mul(buf[k], tw_load<df64>(g.tw, (int64_t)k << (g.lg_P - g.lg_n)));
      scr[k] = c_add(e, t);
      scr[k + h] = c_sub(e, t);
    }
    __syncthreads();
    Z = scr;
  }
  for (int k = threadIdx.x; k <= n / 2; k += BT) {
    const int nk = (n - k) & (n - 1);
    const cplx<df64> tw = k ? twiddle_M<df64>(g.tA, g.tB, g.tws, (int64_t)k << g.twshift)
                            : mk(make_df(1.f, 0.f), df_zero());
    cplx<df64> wk, wnk;
    rfft_post(Z[k], Z[nk], tw, wk, wnk);
    chat[k] = c_scale(wk, s);
    chat[n - k] = c_scale(wnk, s);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- products
template <class T> SSA_D T ldx(const df64* p, int64_t i) { return scal<T>::from_df(p[i]); }

// y = X x (transpose = 0) or X^T x (transpose = 1), one CTA, FFT in shared memory.
template <class T, int MAXE>
SSA_D void cta_matvec(const Geom& g, int transpose, const df64* x, df64* y, const cplx<df64>* chat, cplx<T>* buf) {
  const int n = 1 << g.lg_n;
  for (int t = threadIdx.x; t < n; t += BT) {
    T v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int64_t j = 2 * (int64_t)t + e;
      if (!transpose) v[e] = j < g.K ? ldx<T>(x, g.K - 1 - j) : scal<T>::zero();
      else v[e] = j >= g.M - g.L ? ldx<T>(x, g.M - 1 - j) : scal<T>::zero();
    }
    buf[t] = mk(v[0], v[1]);
  }
  __syncthreads();
  cta_fft<T, BT, MAXE, false>(buf, g.lg_n, 1, g.tw, g.lg_P);
  for (int k = threadIdx.x; k <= n / 2; k += BT) {
    const int nk = (n - k) & (n - 1);
    cplx<T> tw = k ? twiddle_M<T>(g.tA, g.tB, g.tws, (int64_t)k << g.twshift)
                   : mk(scal<T>::from_double(1.0), scal<T>::zero());
    cplx<T> wk, wnk, zk, znk;
    rfft_post(buf[k], buf[nk], tw, wk, wnk);
    cplx<T> pk = mul_spec(wk, chat[k]);
    cplx<T> pnk = mul_spec(wnk, chat[n - k]);
    irfft_pre(pk, pnk, tw, zk, znk);
    buf[k] = zk;
    if (k != 0 && nk != k) buf[nk] = znk;
  }
  __syncthreads();
  cta_fft<T, BT, MAXE, true>(buf, g.lg_n, 1, g.tw, g.lg_P);
  const int64_t off = transpose ? g.M - g.K : 0;
  const int64_t cnt = transpose ? g.K : g.L;
  for (int64_t m = threadIdx.x; m < cnt; m += BT) {
    const int64_t i = off + m;
    const cplx<T> z = buf[i >> 1];
    y[m] = scal<T>::to_df((i & 1) ? z.im : z.re);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- CGS2 in one CTA
// One pass over the basis Q (dim x ncols) in tiles of B_FR = 64 rows:
//   UPD:  w <- w - Q h_in;   PROJ: h_out[c] = Q[:, c] . w (c < ncols), h_out[ncols] = w.w
//   !PROJ: *nrm_out = w.w
// Warp wp owns the columns c = wp + 16m and lane l the rows 2l, 2l+1 of every
// tile, so each lane stages (16-byte asynchronous copies, B_NST tiles deep)
// and reads back only what it copied itself: the basis tiles need no
// barrier.  Under UPD every warp forms the partial row sums of its columns;
// after one barrier eight threads per row add the sixteen partials (pairs,
// then a three-level butterfly: a fixed order) and the first of them writes
// x = w - Q h_in (to shared memory when PROJ follows, and to w).  Under PROJ
// each lane accumulates its columns' products with its two rows of x over all
// tiles in registers; one warp reduction per column at the end.  Rows of w are
// prefetched into registers one tile ahead.
// Two consecutive rows (row even, 16-byte aligned) of a vector this persistent kernel also writes,
// read through L2 (coherent with the kernel's own earlier stores, unlike the read-only path);
// rows >= dim read as 0.
SSA_D float4 ld_pair_l2(const df64* p, int64_t row, int64_t dim) {
  if (row + 1 < dim) return __ldcg(reinterpret_cast<const float4*>(p + row));
  if (row < dim) {
    const float2 a = __ldcg(reinterpret_cast<const float2*>(p + row));
    return make_float4(a.x, a.y, 0.f, 0.f);
  }
  return make_float4(0.f, 0.f, 0.f, 0.f);
}
constexpr int B_W = BT / 32;                    // warps per CTA
constexpr int B_CPW = (B_MAXC + B_W - 1) / B_W;  // basis columns per warp at most
template <bool UPD, bool PROJ>
__device__ __noinline__ void cta_cgs_pass(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim,
                                          const df64* h_in, df64* h_out, df64* nrm_out, df64* stbuf) {
  constexpr int NRED = (UPD && !PROJ) ? 2 : 1;
  static_assert(B_NST * B_MAXC * B_FR + 2 * B_W * B_FR + B_FR <= B_SMEM / 8, "CGS staging exceeds the buffer");
  static_assert(B_W == 16 && BT / 8 == B_FR, "the row reduction pairs 16 warp partials over 8 threads per row");
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int ntiles = (int)((dim + B_FR - 1) / B_FR);
  const int stage_elems = ncols * B_FR;
  df64* red0 = stbuf + B_NST * B_MAXC * B_FR;   // [NRED][B_W][B_FR] row partials
  df64* xs = red0 + 2 * B_W * B_FR;             // [B_FR] updated rows
  __shared__ df64 nred[B_W];
  const int mycols = ncols > wp ? (ncols - wp + B_W - 1) / B_W : 0;  // warp-uniform
  df64 hr[B_CPW];
  dacc acc[B_CPW];
  __syncthreads();  // the buffer's previous users are done
#pragma unroll
  for (int m = 0; m < B_CPW; ++m) {
    hr[m] = (UPD && m < mycols) ? h_in[wp + B_W * m] : df_zero();
    acc[m] = dacc_zero();
  }
  dacc nacc = dacc_zero();
  const df64* qlane = Q + (int64_t)wp * ldq + 2 * lane;
  const int64_t qstep = (int64_t)B_W * ldq;
  auto issue = [&](int stg, int tile) {  // this lane's 16-byte pieces (column c at c * B_FR)
    df64* st = stbuf + stg * stage_elems + wp * B_FR + 2 * lane;
    const int64_t r0 = (int64_t)tile * B_FR;
    const bool ok = r0 + 2 * lane < dim;
#pragma unroll
    for (int m = 0; m < B_CPW; ++m) {
      if (m >= mycols) break;
      cp_async16(st + B_W * m * B_FR, ok ? (const void*)(qlane + m * qstep + r0) : (const void*)Q, ok);
    }
  };
  const int rrow = tid >> 3, rq = tid & 7;  // UPD: eight threads per row
  auto wrow = [&](int tile) -> df64 {
    const int64_t row = (int64_t)tile * B_FR + rrow;
    return row < dim ? w[row] : df_zero();
  };
  auto wpair = [&](int tile) -> float4 { return ld_pair_l2(w, (int64_t)tile * B_FR + 2 * lane, dim); };
  for (int p = 0; p < B_NST - 1; ++p) {
    if (p < ntiles) issue(p, p);
    cp_async_commit();
  }
  df64 wr = df_zero();
  float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ntiles > 0) {
    if (UPD) {
      if (rq == 0) wr = wrow(0);
    } else {
      wv = wpair(0);
    }
  }
  for (int tile = 0; tile < ntiles; ++tile) {
    const int ahead = tile + B_NST - 1;
    if (ahead < ntiles) issue(ahead % B_NST, ahead);
    cp_async_commit();
    df64 wr_n = wr;
    float4 wv_n = wv;
    if (tile + 1 < ntiles) {
      if (UPD) {
        if (rq == 0) wr_n = wrow(tile + 1);
      } else {
        wv_n = wpair(tile + 1);
      }
    }
    cp_async_wait<B_NST - 1>();
    const df64* sl = stbuf + (tile % B_NST) * stage_elems + wp * B_FR + 2 * lane;
    const int64_t r0 = (int64_t)tile * B_FR;
    if (UPD) {
      dacc a0 = dacc_zero(), a1 = dacc_zero();
#pragma unroll
      for (int m = 0; m < B_CPW; ++m) {
        if (m >= mycols) break;
        const float4 v = *reinterpret_cast<const float4*>(sl + B_W * m * B_FR);
        dacc_fma(a0, make_df(v.x, v.y), hr[m]);
        dacc_fma(a1, make_df(v.z, v.w), hr[m]);
      }
      const df64 s0 = dacc_val(a0), s1 = dacc_val(a1);
      df64* rb = red0 + (NRED == 2 ? (tile & 1) : 0) * (B_W * B_FR);
      *reinterpret_cast<float4*>(rb + wp * B_FR + 2 * lane) = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
      __syncthreads();
      {
        df64 sum = df_add(rb[(2 * rq) * B_FR + rrow], rb[(2 * rq + 1) * B_FR + rrow]);
        sum = df_add(sum, shfl_xor_df(sum, 1));
        sum = df_add(sum, shfl_xor_df(sum, 2));
        sum = df_add(sum, shfl_xor_df(sum, 4));
        if (rq == 0) {
          const int64_t row = r0 + rrow;
          const df64 x = row < dim ? df_sub(wr, sum) : df_zero();
          if (PROJ) xs[rrow] = x;
          if (row < dim) w[row] = x;
          dacc_fma(nacc, x, x);
        }
      }
      if (PROJ) __syncthreads();
    }
    if (PROJ) {
      const float4 xv = UPD ? *reinterpret_cast<const float4*>(xs + 2 * lane) : wv;
      const df64 x0 = make_df(xv.x, xv.y), x1 = make_df(xv.z, xv.w);
      if (!UPD && wp == 0) {
        dacc_fma(nacc, x0, x0);
        dacc_fma(nacc, x1, x1);
      }
#pragma unroll
      for (int m = 0; m < B_CPW; ++m) {
        if (m >= mycols) break;
        const float4 v = *reinterpret_cast<const float4*>(sl + B_W * m * B_FR);
        dacc_fma(acc[m], make_df(v.x, v.y), x0);
        dacc_fma(acc[m], make_df(v.z, v.w), x1);
      }
      if ((tile & 15) == 15) {
#pragma unroll
        for (int m = 0; m < B_CPW; ++m) {
          if (m >= mycols) break;
          dacc_norm(acc[m]);
        }
      }
    }
    wr = wr_n;
    wv = wv_n;
  }
  cp_async_wait<0>();
  const df64 nv = warp_sum_df(dacc_val(nacc));
  if (lane == 0) nred[wp] = nv;
  if (PROJ) {
#pragma unroll
    for (int m = 0; m < B_CPW; ++m) {
      if (m >= mycols) break;  // warp-uniform
      const df64 v = warp_sum_df(dacc_val(acc[m]));
      if (lane == 0) h_out[wp + B_W * m] = v;
    }
  }
  __syncthreads();
  if (tid == 0) {
    df64 t = nred[0];
    for (int q = 1; q < B_W; ++q) t = df_add(t, nred[q]);
    if (PROJ) h_out[ncols] = t;
    else *nrm_out = t;
  }
  __syncthreads();
}

// w <- (I - Q Q^T)^2 w; returns w.w (valid in all threads)
// mode: REORTH_ONCE (FP32 products) or REORTH_GATED: after the first
// projection h, with tau > 0, only w - h_l q_l (l the newest column, whose
// coefficient is the bidiagonal coupling) when max_{i<l} |h_i| <= tau ||w'|| and
// ||w||^2 <= SKIP_RATIO ||w'||^2 (the skip test of the single-series
// engine); else the update with a second projection, and the third pass only
// when ||w'||^2 < ||w||^2 / 2 after the first update (Kahan-Parlett).
SSA_D df64 cta_cgs2(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, df64* h1, df64* h2, df64* scal_,
                    df64* stbuf, int mode, double tau) {
  if (ncols > 0) {
    cta_cgs_pass<false, true>(Q, ldq, ncols, w, dim, nullptr, h1, nullptr, stbuf);
    __syncthreads();
    if (mode == REORTH_GATED) {
      if (tau > 0.0) {
        float hm = 0.f;  // every thread reads the same h: a CTA-uniform decision
        for (int i = 0; i < ncols - 1; ++i) hm = fmaxf(hm, fabsf(h1[i].hi));
        const double w2 = df_to_double(h1[ncols]), hl = df_to_double(h1[ncols - 1]);
        const double r2 = w2 - hl * hl;
        if (r2 > 0.0 && (double)hm * (double)hm <= tau * tau * r2 && w2 <= SKIP_RATIO * r2) {
          cta_cgs_pass<true, false>(Q + (int64_t)(ncols - 1) * ldq, ldq, 1, w, dim, h1 + (ncols - 1), nullptr,
                                    scal_, stbuf);
          __syncthreads();
          return *scal_;
        }
      }
      cta_cgs_pass<true, true>(Q, ldq, ncols, w, dim, h1, h2, nullptr, stbuf);
      __syncthreads();
      if (!df_lt(df_scale(h2[ncols], 2.0f), h1[ncols])) return h2[ncols];
      cta_cgs_pass<true, false>(Q, ldq, ncols, w, dim, h2, nullptr, scal_, stbuf);
    } else {
      cta_cgs_pass<true, false>(Q, ldq, ncols, w, dim, h1, nullptr, scal_, stbuf);
    }
  } else {
    cta_cgs_pass<true, false>(Q, ldq, 0, w, dim, h1, nullptr, scal_, stbuf);
  }
  return *scal_;
}

// ---------------------------------------------------------------- Ritz products
// out[:, m] = sum_{i<r} Q[:, i] P[i, m], m < ncol (P column-major, leading dimension ldp)
SSA_D void cta_ritz(const df64* Q, int64_t ldq, int r, const df64* P, int ldp, int ncol, df64* out, int64_t ldo,
                    int64_t dim, df64* Ps) {
  for (int e = threadIdx.x; e < r * ncol; e += BT) {
    const int i = e % r, m = e / r;
    Ps[i * B_MAXC + m] = P[(int64_t)m * ldp + i];
  }
  __syncthreads();
  for (int m0 = 0; m0 < ncol; m0 += 16) {
    for (int64_t row = threadIdx.x; row < dim; row += BT) {
      dacc acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = dacc_zero();
      for (int i = 0; i < r; ++i) {
        const df64 q = Q[(int64_t)i * ldq + row];
        const df64* pr = Ps + i * B_MAXC + m0;
#pragma unroll
        for (int j = 0; j < 16; ++j) dacc_fma(acc[j], q, pr[j]);
        if ((i & 31) == 31) {
#pragma unroll
          for (int j = 0; j < 16; ++j) dacc_norm(acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (m0 + j < ncol) out[(int64_t)(m0 + j) * ldo + row] = dacc_val(acc[j]);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- the kernel
template <class T, int MAXE>
__global__ void __launch_bounds__(BT, 1) k_batch_ssa(BCtx cx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* fbuf = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<df64>* dbuf = reinterpret_cast<cplx<df64>*>(smem_raw);
  df64* stbuf = reinterpret_cast<df64*>(smem_raw);
  __shared__ int s_item;
  __shared__ df64 h1[B_MAXC + 2], h2[B_MAXC + 2];
  __shared__ df64 sc_nrm, est;
  __shared__ int conv;
  __shared__ unsigned status;
  const Slot sl = carve(cx, blockIdx.x);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(cx.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= cx.nseries) break;
    const int si = cx.order[item];
    const BSeries S = cx.ser[si];
    Geom g{};
    g.N = S.N;
    g.L = S.Lw;
    g.K = S.Kw;
    g.M = (int64_t)2 << S.lg_n;
    g.lg_n = S.lg_n;
    g.tw = cx.tw;
    g.lg_P = cx.lg_P;
    g.tA = cx.tA;
    g.tB = cx.tB;
    g.tws = cx.tws;
    g.twshift = cx.lg_Mmax - (S.lg_n + 1);
    const double* f = cx.f + S.f_off;
    const int d = S.d, kk = S.kk, k = S.k;
    const int64_t Lw = S.Lw, Kw = S.Kw, ldu = cx.ldu, ldv = cx.ldv;
    const int ldb = B_MAXC;
    const uint64_t seed = cx.seed;  // same draws alone and in any batch
    const int reorth = cx.precision == SSA_PREC_F32C ? REORTH_ONCE : REORTH_GATED;
    // spectrum
    const int fexp = cta_series_exp(f, S.N);
    cta_spectrum(g, f, ldexp(1.0, -fexp), sl.chat, sl.fscr, dbuf);
    // clear the projected matrix; state
    for (int e = threadIdx.x; e < ldb * ldb; e += BT) sl.B[e] = df_zero();
    if (threadIdx.x == 0) {
      est = df_zero();
      status = 0u;
      conv = 0;
    }
    __syncthreads();
    int cur = 0;
    df64* U = sl.U[0];
    df64* V = sl.V[0];
    uint64_t stream_id = 0;
    int matvecs = 0;
    // normalise w into qcol with breakdown replacement (coefficient -> *bentry)
    auto normalize = [&](df64* w, int64_t dim, df64 nrm2, df64* Qb, int64_t ldq, int ncols, df64* bentry) {
      df64 beta = df_sqrt(nrm2);
      const bool good = beta.hi > 1e-14f * est.hi && beta.hi > 0.f && isfinite(beta.hi);
      if (!isfinite(beta.hi) && threadIdx.x == 0) status |= SSA_DEV_NONFINITE;
      df64* qcol = Qb + (int64_t)ncols * ldq;
      if (good) {
        const df64 inv = df_div(make_df(1.f, 0.f), beta);
        for (int64_t i = threadIdx.x; i < dim; i += BT) qcol[i] = df_mul(w[i], inv);
        __syncthreads();
        if (threadIdx.x == 0) {
          *bentry = beta;
          if (df_gt(beta, est)) est = beta;
        }
      } else {
        for (int64_t i = threadIdx.x; i < dim; i += BT) w[i] = sm64_uniform_pm1(seed, stream_id, i);
        __syncthreads();
        const df64 n2 = cta_cgs2(Qb, ldq, ncols, w, dim, h1, h2, &sc_nrm, stbuf, reorth, cx.skip_tau);
        const df64 nb = df_sqrt(n2);
        const bool alive = ncols < dim && nb.hi > 1e-6f * sqrtf((float)dim / 3.f);
        const df64 inv = alive ? df_div(make_df(1.f, 0.f), nb) : df_zero();
        for (int64_t i = threadIdx.x; i < dim; i += BT) qcol[i] = df_mul(w[i], inv);
        __syncthreads();
        if (threadIdx.x == 0) {
          *bentry = df_zero();
          status |= SSA_DEV_BREAKDOWN;
        }
      }
      __syncthreads();
    };
    // p_0
    for (int64_t i = threadIdx.x; i < Lw; i += BT) sl.y[i] = sm64_uniform_pm1(seed, stream_id, i);
    ++stream_id;
    __syncthreads();
    {
      const df64 n2 = cta_cgs2(U, ldu, 0, sl.y, Lw, h1, h2, &sc_nrm, stbuf, reorth, cx.skip_tau);
      normalize(sl.y, Lw, n2, U, ldu, 0, &sl.T[0]);
    }
    int r = 1, c = 0;
    auto side = [&](bool vside) {
      df64* Qb = vside ? V : U;
      const int64_t ldq = vside ? ldv : ldu;
      const int64_t dim = vside ? Kw : Lw;
      const int ncols = vside ? c : r;
      const df64* src = vside ? U + (int64_t)(r - 1) * ldu : V + (int64_t)(c - 1) * ldv;
      df64* bentry = vside ? sl.B + (int64_t)(r - 1) * ldb + c : sl.B + (int64_t)r * ldb + (c - 1);
      cta_matvec<T, MAXE>(g, vside ? 1 : 0, src, sl.y, sl.chat, fbuf);
      ++matvecs;
      const df64 n2 = cta_cgs2(Qb, ldq, ncols, sl.y, dim, h1, h2, &sc_nrm, stbuf, reorth, cx.skip_tau);
      normalize(sl.y, dim, n2, Qb, ldq, ncols, bentry);
      ++stream_id;
      if (vside) ++c;
      else ++r;
    };
    int restarts = 0;
    side(true);
    for (;;) {
      while (c < d + 1) {
        side(false);
        side(true);
      }
      const int cp = c - 1;
      const int cc = cp + (cp & 1);
      const bool pre = cp >= 16 && ((size_t)r * cp + (size_t)cp * cp) * 4 <= (size_t)B_SMEM;
      if (pre) {
        float* A32 = reinterpret_cast<float*>(smem_raw);
        svd_precondition_body<BT>(sl.B, ldb, r, cp, sl.A, sl.W, sl.T, cc, PRE_SWEEPS, 2e-6f, A32, A32 + r * cp);
        __syncthreads();
      }
      // the FFT buffer is idle during the projected SVD: stage A and W there
      svd_jacobi_body<BT>(sl.B, ldb, r, cp, sl.A, sl.W, cc, sl.sigma, sl.P, sl.Q, sl.resid, sl.sigma_d, k, cx.tol,
                          &conv, &est, &status, 60, 1e-13f, pre ? 1 : 0, reinterpret_cast<df64*>(smem_raw));
      __syncthreads();
      const int converged = conv;
      __syncthreads();
      if (converged || restarts >= cx.max_restarts || kk >= cp) break;
      // thick restart
      const int nxt = cur ^ 1;
      cta_ritz(U, ldu, r, sl.P, r, kk, sl.U[nxt], ldu, Lw, stbuf);
      cta_ritz(V, ldv, cp, sl.Q, cp, kk, sl.V[nxt], ldv, Kw, stbuf);
      for (int64_t i = threadIdx.x; i < Kw; i += BT) sl.V[nxt][(int64_t)kk * ldv + i] = V[(int64_t)cp * ldv + i];
      {
        const df64 ar = sl.B[(int64_t)(r - 1) * ldb + cp];
        __syncthreads();
        for (int e = threadIdx.x; e < ldb * ldb; e += BT) sl.B[e] = df_zero();
        __syncthreads();
        for (int i = threadIdx.x; i < kk; i += BT) {
          sl.B[(int64_t)i * ldb + i] = sl.sigma[i];
          sl.B[(int64_t)i * ldb + kk] = df_mul(ar, sl.P[(int64_t)i * r + (r - 1)]);
        }
      }
      __syncthreads();
      cur = nxt;
      U = sl.U[cur];
      V = sl.V[cur];
      r = kk;
      c = kk + 1;
      ++restarts;
    }
    // Ritz vectors of the k wanted triples into the other buffers
    const int cp = c - 1;
    df64* Uf = sl.U[cur ^ 1];
    df64* Vf = sl.V[cur ^ 1];
    cta_ritz(U, ldu, r, sl.P, r, k, Uf, ldu, Lw, stbuf);
    cta_ritz(V, ldv, cp, sl.Q, cp, k, Vf, ldv, Kw, stbuf);
    // sign rule on the user's left vectors, then doubles in user orientation
    const df64* Uu = S.transposed ? Vf : Uf;
    const int64_t ldus = S.transposed ? ldv : ldu;
    const int64_t Lu = S.transposed ? Kw : Lw;
    __shared__ float sb[BT / 32];
    __shared__ int64_t sidx[BT / 32];
    __shared__ int sgn[B_MAXC];
    for (int j = 0; j < k; ++j) {
      const df64* u = Uu + (int64_t)j * ldus;
      df64 best = make_df(-1.f, 0.f);
      int64_t bi = 0;
      for (int64_t i = threadIdx.x; i < Lu; i += BT) {
        const df64 a = df_abs(u[i]);
        if (df_gt(a, best)) { best = a; bi = i; }
      }
      for (int m = 16; m; m >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, best.hi, m);
        const float ol = __shfl_xor_sync(0xffffffffu, best.lo, m);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, m);
        const df64 o = make_df(oh, ol);
        if (df_gt(o, best) || (o.hi == best.hi && o.lo == best.lo && oi < bi)) { best = o; bi = oi; }
      }
      if ((threadIdx.x & 31) == 0) { sb[threadIdx.x >> 5] = best.hi + best.lo; sidx[threadIdx.x >> 5] = bi; }
      __syncthreads();
      if (threadIdx.x == 0) {
        float bv = -1.f;
        int64_t bj = 0;
        for (int wv = 0; wv < BT / 32; ++wv)
          if (sb[wv] > bv || (sb[wv] == bv && sidx[wv] < bj)) { bv = sb[wv]; bj = sidx[wv]; }
        sgn[j] = u[bj].hi < 0.f ? -1 : 1;
      }
      __syncthreads();
    }
    double* oU = cx.out_U + S.out_u;
    double* oV = cx.out_V + S.out_v;
    const df64* srcU = S.transposed ? Vf : Uf;
    const df64* srcV = S.transposed ? Uf : Vf;
    const int64_t ldsu = S.transposed ? ldv : ldu, ldsv = S.transposed ? ldu : ldv;
    for (int64_t e = threadIdx.x; e < S.L * (int64_t)k; e += BT) {
      const int64_t j = e / S.L, i = e - j * S.L;
      oU[e] = df_to_double(srcU[j * ldsu + i]) * sgn[j];
    }
    for (int64_t e = threadIdx.x; e < S.K * (int64_t)k; e += BT) {
      const int64_t j = e / S.K, i = e - j * S.K;
      oV[e] = df_to_double(srcV[j * ldsv + i]) * sgn[j];
    }
    const double unscale = ldexp(1.0, fexp);  // back to the caller's units
    for (int j = threadIdx.x; j < k; j += BT) {
      cx.out_sigma[S.out_s + j] = sl.sigma_d[j] * unscale;
      cx.out_resid[S.out_s + j] = sl.resid[j] * unscale;
    }
    if (threadIdx.x == 0) {
      cx.out_info[4 * si + 0] = conv;
      cx.out_info[4 * si + 1] = restarts;
      cx.out_info[4 * si + 2] = matvecs;
      cx.out_info[4 * si + 3] = (int)status;
    }
    __syncthreads();
    (void)cp;
  }
}

// ---------------------------------------------------------------- refinement
// sigma_j <- u_j^T (X v_j) with native-FP64 FFT products (n <= 8192, one CTA
// per series), then the triples are re-sorted if two nearly equal values
// swapped.  Runs after k_batch_ssa and reuses its slots: the spectrum goes
// to the slot's spectrum area, column permutations use its V basis area.
struct BRefine {
  const cplx<double>* tw;
  const cplx<double>* tA;
  const cplx<double>* tB;
  int* next;
};

__global__ void __launch_bounds__(BT) k_batch_refine(BCtx cx, BRefine rf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<double>* buf = reinterpret_cast<cplx<double>*>(smem_raw);
  __shared__ int s_item;
  __shared__ double red[BT / 32];
  __shared__ double sg[B_MAXC];
  __shared__ int perm[B_MAXC];
  __shared__ int sorted;
  const Slot sl = carve(cx, blockIdx.x);
  cplx<double>* chat = reinterpret_cast<cplx<double>*>(sl.chat);
  double* tmp = reinterpret_cast<double*>(sl.V[0]);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(rf.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= cx.nseries) break;
    const int si = cx.order[item];
    const BSeries S = cx.ser[si];
    Geom g{};
    g.N = S.N;
    g.L = S.Lw;
    g.K = S.Kw;
    g.M = (int64_t)2 << S.lg_n;
    g.lg_n = S.lg_n;
    g.tw64 = rf.tw;
    g.lg_P = cx.lg_P;
    g.tA64 = rf.tA;
    g.tB64 = rf.tB;
    g.tws = cx.tws;
    g.twshift = cx.lg_Mmax - (S.lg_n + 1);
    const double* f = cx.f + S.f_off;
    const int n = 1 << g.lg_n;
    const cplx<double> one = mk(1.0, 0.0);
    // spectrum of the circulant column, scaled by 1/(4n)
    for (int t = threadIdx.x; t < n; t += BT) buf[t] = mk(circ(g, f, 2 * (int64_t)t), circ(g, f, 2 * (int64_t)t + 1));
    __syncthreads();
    cta_fft<double, BT, 8192, false>(buf, g.lg_n, 1, g.tw64, g.lg_P);
    const double sc = 0.5 / (4.0 * (double)n);
    for (int kx = threadIdx.x; kx <= n / 2; kx += BT) {
      const int nk = (n - kx) & (n - 1);
      const cplx<double> tw = kx ? twiddle_M<double>(g.tA64, g.tB64, g.tws, (int64_t)kx << g.twshift) : one;
      cplx<double> wk, wnk;
      rfft_post(buf[kx], buf[nk], tw, wk, wnk);
      chat[kx] = mk(wk.re * sc, wk.im * sc);
      chat[n - kx] = mk(wnk.re * sc, wnk.im * sc);
    }
    __syncthreads();
    const double* Ui = cx.out_U + S.out_u;  // user orientation, signs applied to u and v alike
    const double* Vi = cx.out_V + S.out_v;
    const int64_t ldUi = S.L, ldVi = S.K;
    if (S.transposed) {  // working orientation: u in the user's V, v in the user's U
      const double* t = Ui; Ui = Vi; Vi = t;
    }
    const int64_t ldu_w = S.transposed ? ldVi : ldUi, ldv_w = S.transposed ? ldUi : ldVi;
    for (int j = 0; j < S.k; ++j) {
      const double* v = Vi + (int64_t)j * ldv_w;
      const double* u = Ui + (int64_t)j * ldu_w;
      for (int t = threadIdx.x; t < n; t += BT) {
        const int64_t j0 = 2 * (int64_t)t, j1 = j0 + 1;
        buf[t] = mk(j0 < g.K ? v[g.K - 1 - j0] : 0.0, j1 < g.K ? v[g.K - 1 - j1] : 0.0);
      }
      __syncthreads();
      cta_fft<double, BT, 8192, false>(buf, g.lg_n, 1, g.tw64, g.lg_P);
      for (int kx = threadIdx.x; kx <= n / 2; kx += BT) {
        const int nk = (n - kx) & (n - 1);
        const cplx<double> tw = kx ? twiddle_M<double>(g.tA64, g.tB64, g.tws, (int64_t)kx << g.twshift) : one;
        cplx<double> wk, wnk, zk, znk;
        rfft_post(buf[kx], buf[nk], tw, wk, wnk);
        irfft_pre(c_mul(wk, chat[kx]), c_mul(wnk, chat[n - kx]), tw, zk, znk);
        buf[kx] = zk;
        if (kx != 0 && nk != kx) buf[nk] = znk;
      }
      __syncthreads();
      cta_fft<double, BT, 8192, true>(buf, g.lg_n, 1, g.tw64, g.lg_P);
      double acc = 0.0;
      for (int64_t m = threadIdx.x; m < g.L; m += BT) {
        const cplx<double> z = buf[m >> 1];
        acc = fma(u[m], (m & 1) ? z.im : z.re, acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < BT / 32; ++w) t += red[w];
        sg[j] = t;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {  // stable insertion sort, descending
      sorted = 1;
      for (int j = 0; j < S.k; ++j) perm[j] = j;
      for (int j = 1; j < S.k; ++j) {
        const int pj = perm[j];
        int q = j;
        while (q > 0 && sg[perm[q - 1]] < sg[pj]) {
          perm[q] = perm[q - 1];
          --q;
        }
        perm[q] = pj;
        if (q != j) sorted = 0;
      }
    }
    __syncthreads();
    double* osig = cx.out_sigma + S.out_s;
    double* ores = cx.out_resid + S.out_s;
    if (sorted) {
      for (int j = threadIdx.x; j < S.k; j += BT) osig[j] = sg[j];
    } else {
      for (int j = threadIdx.x; j < S.k; j += BT) tmp[j] = ores[j];
      __syncthreads();
      for (int j = threadIdx.x; j < S.k; j += BT) {
        osig[j] = sg[perm[j]];
        ores[j] = tmp[perm[j]];
      }
      __syncthreads();
      double* cols[2] = {cx.out_U + S.out_u, cx.out_V + S.out_v};
      const int64_t lens[2] = {S.L, S.K};
      for (int a = 0; a < 2; ++a) {
        const int64_t tot = lens[a] * S.k;
        for (int64_t e = threadIdx.x; e < tot; e += BT) tmp[e] = cols[a][e];
        __syncthreads();
        for (int64_t e = threadIdx.x; e < tot; e += BT) {
          const int64_t j = e / lens[a], i = e - j * lens[a];
          cols[a][e] = tmp[(int64_t)perm[j] * lens[a] + i];
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) cx.out_info[4 * si + 2] += S.k;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- grouped Hankelization
// For every (series, group): g = irFFT(sum_{j in group} sigma_j rFFT(u'_j) . rFFT(v'_j)) / counts
// (Algorithm 4 summed over the group, with the division by the antidiagonal
// counts of section 5).  One persistent CTA per item at a time; the u'
// spectrum and the group's accumulator (df64) live in the CTA's global
// scratch, the FFTs in shared memory.
struct BHCtx {
  const BSeries* ser;
  int nseries, m;
  const double *U, *V, *sigma;
  const int *grp_off, *grp_idx;
  double* out;
  const int64_t* out_off;  // per series: start of its m x N block in out
  const cplx<df64>* tw;
  int lg_P;
  const cplx<df64>* tA;
  const cplx<df64>* tB;
  int tws, lg_Mmax;
  cplx<df64>* scratch;
  int64_t ld_scr;  // 2 (nmax + 1) per CTA
  int* next;
};

template <class T, int MAXE>
SSA_D void cta_rfft_pad(const Geom& g, const double* x, int64_t len, cplx<T>* buf) {
  const int n = 1 << g.lg_n;
  for (int t = threadIdx.x; t < n; t += BT) {
    const int64_t j = 2 * (int64_t)t;
    buf[t] = mk(j < len ? scal<T>::from_double(x[j]) : scal<T>::zero(),
                j + 1 < len ? scal<T>::from_double(x[j + 1]) : scal<T>::zero());
  }
  __syncthreads();
  cta_fft<T, BT, MAXE, false>(buf, g.lg_n, 1, g.tw, g.lg_P);
}

template <class T, int MAXE>
__global__ void __launch_bounds__(BT, 1) k_batch_hankel(BHCtx cx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  __shared__ int s_item;
  cplx<df64>* su = cx.scratch + (int64_t)blockIdx.x * cx.ld_scr;
  cplx<df64>* acc = su + cx.ld_scr / 2;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(cx.next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= cx.nseries * cx.m) break;
    const int si = item / cx.m, grp = item - si * cx.m;
    const BSeries S = cx.ser[si];
    Geom g{};
    g.N = S.N;
    g.L = S.L;
    g.K = S.K;
    g.M = (int64_t)2 << S.lg_n;
    g.lg_n = S.lg_n;
    g.tw = cx.tw;
    g.lg_P = cx.lg_P;
    g.tA = cx.tA;
    g.tB = cx.tB;
    g.tws = cx.tws;
    g.twshift = cx.lg_Mmax - (S.lg_n + 1);
    const int n = 1 << g.lg_n;
    // sigma scaled by 2^-e (e of the series' largest sigma) into double-float range, the
    // output scaled back by 2^e: exact, whatever the units of the series
    int e = 0;
    if (cx.sigma[S.out_s] > 0.0) frexp(cx.sigma[S.out_s], &e);
    const double sg_scale = ldexp(1.0, -e);
    for (int k = threadIdx.x; k <= n; k += BT) acc[k] = mk(df_zero(), df_zero());
    for (int ii = cx.grp_off[grp]; ii < cx.grp_off[grp + 1]; ++ii) {
      const int j = cx.grp_idx[ii];
      const double* u = cx.U + S.out_u + (int64_t)j * S.L;
      const double* v = cx.V + S.out_v + (int64_t)j * S.K;
      const df64 sg = df_from_double(cx.sigma[S.out_s + j] * sg_scale);
      cta_rfft_pad<T, MAXE>(g, u, S.L, buf);
      for (int k = threadIdx.x; k <= n / 2; k += BT) {
        const int nk = (n - k) & (n - 1);
        const cplx<T> tw = k ? twiddle_M<T>(g.tA, g.tB, g.tws, (int64_t)k << g.twshift)
                             : mk(scal<T>::from_double(1.0), scal<T>::zero());
        cplx<T> wk, wnk;
        rfft_post(buf[k], buf[nk], tw, wk, wnk);
        su[k] = mk(scal<T>::to_df(wk.re), scal<T>::to_df(wk.im));
        su[n - k] = mk(scal<T>::to_df(wnk.re), scal<T>::to_df(wnk.im));
      }
      __syncthreads();
      cta_rfft_pad<T, MAXE>(g, v, S.K, buf);
      for (int k = threadIdx.x; k <= n / 2; k += BT) {
        const int nk = (n - k) & (n - 1);
        const cplx<T> tw = k ? twiddle_M<T>(g.tA, g.tB, g.tws, (int64_t)k << g.twshift)
                             : mk(scal<T>::from_double(1.0), scal<T>::zero());
        cplx<T> wk, wnk;
        rfft_post(buf[k], buf[nk], tw, wk, wnk);
        const cplx<df64> a = c_mul(su[k], mk(scal<T>::to_df(wk.re), scal<T>::to_df(wk.im)));
        acc[k] = c_add(acc[k], mk(df_mul(a.re, sg), df_mul(a.im, sg)));
        if (n - k != k) {
          const cplx<df64> b = c_mul(su[n - k], mk(scal<T>::to_df(wnk.re), scal<T>::to_df(wnk.im)));
          acc[n - k] = c_add(acc[n - k], mk(df_mul(b.re, sg), df_mul(b.im, sg)));
        }
      }
      __syncthreads();
    }
    // inverse: acc holds 4 sum sigma U V; irfft_pre doubles it; the inverse FFT scales by n
    for (int k = threadIdx.x; k <= n / 2; k += BT) {
      const int nk = (n - k) & (n - 1);
      const cplx<T> tw = k ? twiddle_M<T>(g.tA, g.tB, g.tws, (int64_t)k << g.twshift)
                           : mk(scal<T>::from_double(1.0), scal<T>::zero());
      const cplx<T> pk = mk(scal<T>::from_df(acc[k].re), scal<T>::from_df(acc[k].im));
      const cplx<T> pnk = mk(scal<T>::from_df(acc[n - k].re), scal<T>::from_df(acc[n - k].im));
      cplx<T> zk, znk;
      irfft_pre(pk, pnk, tw, zk, znk);
      buf[k] = zk;
      if (k != 0 && nk != k) buf[nk] = znk;
    }
    __syncthreads();
    cta_fft<T, BT, MAXE, true>(buf, g.lg_n, 1, g.tw, g.lg_P);
    double* o = cx.out + cx.out_off[si] + (int64_t)grp * S.N;
    const double scale = ldexp(1.0, e) / (8.0 * (double)n);
    const int64_t mn = S.L < S.K ? S.L : S.K;
    for (int64_t t = threadIdx.x; t < S.N; t += BT) {
      const cplx<T> z = buf[t >> 1];
      const double p = df_to_double(scal<T>::to_df((t & 1) ? z.im : z.re));
      int64_t c = t + 1;
      if (S.N - t < c) c = S.N - t;
      if (mn < c) c = mn;
      o[t] = p * scale / (double)c;
    }
    __syncthreads();
  }
}

}  // namespace ssa

using namespace ssa;

// ---------------------------------------------------------------- host API
struct ssa_batch_s {
  int nseries = 0;
  std::vector<BSeries> ser;
  std::vector<int> info;  // 4 per series
  double *U = nullptr, *V = nullptr, *sigma = nullptr, *resid = nullptr;
  int64_t totU = 0, totV = 0, totS = 0;
  cudaStream_t stream = nullptr;  // outputs are stream-ordered allocations on this stream
  int precision = SSA_PREC_F64;
  int lg_Mmax = 2;
  // launch state kept for repeated runs (plan/run/wait): device tables, series
  // table, work order, queue counters, per-series info, CTA slots
  cplx<df64> *dtw = nullptr, *dA = nullptr, *dB = nullptr;
  cplx<double> *dtw64 = nullptr, *dA64 = nullptr, *dB64 = nullptr;
  BSeries* dser = nullptr;
  int *dorder = nullptr, *dnext = nullptr, *dinfo = nullptr;
  char* slots = nullptr;
  double* fbuf = nullptr;  // device copy of host series
  int64_t ftot = 0;
  int nslots = 0;
  bool refine = false;
  BCtx cx{};
};

static int bfail(int code, const char* msg) {
  host_set_error(msg);
  return code;
}
#define BCK(x)                                                         \
  do {                                                                 \
    cudaError_t e_ = (x);                                              \
    if (e_ != cudaSuccess) {                                           \
      char m_[256];                                                    \
      std::snprintf(m_, sizeof m_, "%s: %s", #x, cudaGetErrorString(e_)); \
      return bfail(e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA, m_); \
    }                                                                  \
  } while (0)

static bool b_on_device(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class X>
static int to_host(const X* p, size_t n, std::vector<X>& out) {
  out.resize(n);
  if (b_on_device(p)) BCK(cudaMemcpy(out.data(), p, n * sizeof(X), cudaMemcpyDeviceToHost));
  else std::memcpy(out.data(), p, n * sizeof(X));
  return SSA_OK;
}

static cplx<double> b_tw64(int64_t m, int64_t P) {
  m %= P;
  const long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)P;
  return mk((double)cosl(th), -(double)sinl(th));
}

static cplx<df64> b_tw(int64_t m, int64_t P) {
  m %= P;
  const long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)P;
  cplx<df64> z;
  z.re = df_from_double((double)cosl(th));
  z.im = df_from_double(-(double)sinl(th));
  return z;
}

// Validate the series, order them, build the twiddle tables and allocate
// everything a run needs (no series data yet).
static int batch_build(int nseries, const int64_t* offsets, const int64_t* Ls, const int32_t* ks,
                       const ssa_opts_t* opts, ssa_batch_t* out) {
  if (!out) return bfail(SSA_EINVAL, "out is NULL");
  *out = nullptr;
  if (nseries < 1 || !offsets || !Ls || !ks) return bfail(SSA_EINVAL, "need nseries >= 1 and non-NULL arrays");
  ssa_opts_t o;
  if (opts) o = *opts;
  else ssa_default_opts(&o);
  if (o.precision != SSA_PREC_F64 && o.precision != SSA_PREC_F32C) return bfail(SSA_EINVAL, "unknown precision");
  const int64_t nmax_allowed = o.precision == SSA_PREC_F32C ? 32768 : 16384;
  // native-FP64 Rayleigh quotients need N <= 16384 (the double FFT fits one CTA)
  if (o.refine != SSA_REFINE_OFF && o.refine != SSA_REFINE_ON) return bfail(SSA_EINVAL, "unknown refine mode");
  if (!(o.reorth_skip >= 0.0 && o.reorth_skip < 1e-3)) return bfail(SSA_EINVAL, "reorth_skip must be in [0, 1e-3)");
  const bool refine = o.refine == SSA_REFINE_ON;
  std::vector<int64_t> off, L;
  std::vector<int32_t> kv;
  int rc = to_host(offsets, (size_t)nseries + 1, off);
  if (rc) return rc;
  rc = to_host(Ls, (size_t)nseries, L);
  if (rc) return rc;
  rc = to_host(ks, (size_t)nseries, kv);
  if (rc) return rc;
  if (off[0] != 0) return bfail(SSA_EINVAL, "offsets[0] must be 0");
  ssa_batch_s* b = new (std::nothrow) ssa_batch_s();
  if (!b) return SSA_ENOMEM;
  b->nseries = nseries;
  b->ser.resize(nseries);
  int64_t ldu = 4, ldv = 4;
  int lgMmax = 2, nmax = 2;
  for (int i = 0; i < nseries; ++i) {
    BSeries& S = b->ser[i];
    S.f_off = off[i];
    S.N = off[i + 1] - off[i];
    S.L = L[i];
    S.K = S.N - S.L + 1;
    char msg[160];
    if (S.N <= 2 || S.N > (refine ? 16384 : nmax_allowed) || S.L <= 1 || S.L >= S.N) {
      std::snprintf(msg, sizeof msg, "series %d: need 2 < N <= %lld and 1 < L < N", i,
                    (long long)(refine ? 16384 : nmax_allowed));
      delete b;
      return bfail(SSA_EINVAL, msg);
    }
    S.transposed = S.L > S.K;
    S.Lw = S.transposed ? S.K : S.L;
    S.Kw = S.transposed ? S.L : S.K;
    S.k = kv[i];
    if (S.k < 1 || S.k > S.Lw) {
      std::snprintf(msg, sizeof msg, "series %d: need 1 <= k <= min(L, K)", i);
      delete b;
      return bfail(SSA_EINVAL, msg);
    }
    int d = o.krylov_dim > 0 ? o.krylov_dim : b_krylov_dim(S.Lw, S.k);
    if (d > S.Lw) d = (int)S.Lw;
    if (d < S.k) d = S.k;
    if (d > B_MAXD) {
      std::snprintf(msg, sizeof msg, "series %d: Krylov dimension %d above the batched limit %d", i, d, B_MAXD);
      delete b;
      return bfail(SSA_EINVAL, msg);
    }
    int kk = o.keep > 0 ? o.keep : S.k + (d - S.k + 4) / 5;
    if (kk > d - 1) kk = d - 1;
    if (kk < S.k) kk = S.k;
    S.d = d;
    S.kk = kk;
    int64_t M = 4;
    while (M < S.N) M *= 2;
    int lg = 0;
    while (((int64_t)1 << lg) < M) ++lg;
    S.lg_n = lg - 1;
    lgMmax = std::max(lgMmax, lg);
    nmax = std::max(nmax, (int)(M / 2));
    ldu = std::max(ldu, (S.Lw + 3) / 4 * 4);
    ldv = std::max(ldv, (S.Kw + 3) / 4 * 4);
    S.out_u = b->totU;
    S.out_v = b->totV;
    S.out_s = b->totS;
    b->totU += S.L * S.k;
    b->totV += S.K * S.k;
    b->totS += S.k;
  }
  // work order: largest estimated cost first
  std::vector<int> order(nseries);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c2) {
    const double ca = (double)b->ser[a].N * b->ser[a].d * b->ser[a].d;
    const double cb = (double)b->ser[c2].N * b->ser[c2].d * b->ser[c2].d;
    return ca > cb;
  });
  b->lg_Mmax = lgMmax;
  // twiddle tables for the largest transform
  const int64_t Mmax = (int64_t)1 << lgMmax;
  const int lg_P = lgMmax - 1;
  const int64_t P = (int64_t)1 << lg_P;
  const int tws = (lgMmax + 1) / 2;
  const int64_t nA = Mmax >> tws, nB = (int64_t)1 << tws;
  std::vector<cplx<df64>> htw(P), hA(nA), hB(nB);
  for (int64_t m = 0; m < P; ++m) htw[m] = b_tw(m, P);
  for (int64_t m = 0; m < nA; ++m) hA[m] = b_tw(m << tws, Mmax);
  for (int64_t m = 0; m < nB; ++m) hB[m] = b_tw(m, Mmax);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o.stream);
  b->stream = s;
  b->precision = o.precision;
  int dev = 0, sms = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nslots = std::min(sms, nseries);
  const int64_t sbytes = slot_bytes_for(ldu, ldv, nmax);
  // device buffers (owned by the batch)
#define BCK2(x)                                                        \
  do {                                                                 \
    cudaError_t e_ = (x);                                              \
    if (e_ != cudaSuccess) {                                           \
      char m_[256];                                                    \
      std::snprintf(m_, sizeof m_, "%s: %s", #x, cudaGetErrorString(e_)); \
      ssa_batch_destroy(b);                                            \
      return bfail(e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA, m_); \
    }                                                                  \
  } while (0)
  b->nslots = nslots;
  b->refine = refine;
  b->ftot = off[nseries];
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dtw), P * sizeof(cplx<df64>), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dA), nA * sizeof(cplx<df64>), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dB), nB * sizeof(cplx<df64>), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dser), nseries * sizeof(BSeries), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dorder), nseries * sizeof(int), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dnext), 2 * sizeof(int), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dinfo), 4 * (size_t)nseries * sizeof(int), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->slots), (size_t)nslots * sbytes, s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->U), std::max<int64_t>(b->totU, 1) * sizeof(double), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->V), std::max<int64_t>(b->totV, 1) * sizeof(double), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->sigma), std::max<int64_t>(b->totS, 1) * sizeof(double), s));
  BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->resid), std::max<int64_t>(b->totS, 1) * sizeof(double), s));
  BCK2(cudaMemcpyAsync(b->dtw, htw.data(), P * sizeof(cplx<df64>), cudaMemcpyHostToDevice, s));
  BCK2(cudaMemcpyAsync(b->dA, hA.data(), nA * sizeof(cplx<df64>), cudaMemcpyHostToDevice, s));
  BCK2(cudaMemcpyAsync(b->dB, hB.data(), nB * sizeof(cplx<df64>), cudaMemcpyHostToDevice, s));
  BCK2(cudaMemcpyAsync(b->dser, b->ser.data(), nseries * sizeof(BSeries), cudaMemcpyHostToDevice, s));
  BCK2(cudaMemcpyAsync(b->dorder, order.data(), nseries * sizeof(int), cudaMemcpyHostToDevice, s));
  if (refine) {
    std::vector<cplx<double>> h64(std::max(P, std::max(nA, nB)));
    BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dtw64), P * sizeof(cplx<double>), s));
    BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dA64), nA * sizeof(cplx<double>), s));
    BCK2(cudaMallocAsync(reinterpret_cast<void**>(&b->dB64), nB * sizeof(cplx<double>), s));
    for (int64_t m = 0; m < P; ++m) h64[m] = b_tw64(m, P);
    BCK2(cudaMemcpyAsync(b->dtw64, h64.data(), P * sizeof(cplx<double>), cudaMemcpyHostToDevice, s));
    for (int64_t m = 0; m < nA; ++m) h64[m] = b_tw64(m << tws, Mmax);
    BCK2(cudaMemcpyAsync(b->dA64, h64.data(), nA * sizeof(cplx<double>), cudaMemcpyHostToDevice, s));
    for (int64_t m = 0; m < nB; ++m) h64[m] = b_tw64(m, Mmax);
    BCK2(cudaMemcpyAsync(b->dB64, h64.data(), nB * sizeof(cplx<double>), cudaMemcpyHostToDevice, s));
  }
  BCK2(cudaFuncSetAttribute(k_batch_ssa<float, 16384>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM));
  BCK2(cudaFuncSetAttribute(k_batch_ssa<df64, 8192>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM));
  BCK2(cudaFuncSetAttribute(k_batch_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM));
  BCtx& cx = b->cx;
  cx.ser = b->dser;
  cx.nseries = nseries;
  cx.order = b->dorder;
  cx.next = b->dnext;
  cx.f = nullptr;
  cx.out_U = b->U;
  cx.out_V = b->V;
  cx.out_sigma = b->sigma;
  cx.out_resid = b->resid;
  cx.out_info = b->dinfo;
  cx.tw = b->dtw;
  cx.lg_P = lg_P;
  cx.tA = b->dA;
  cx.tB = b->dB;
  cx.tws = tws;
  cx.lg_Mmax = lgMmax;
  cx.slots = b->slots;
  cx.slot_bytes = sbytes;
  cx.ldu = ldu;
  cx.ldv = ldv;
  cx.nmax = nmax;
  cx.precision = o.precision;
  cx.skip_tau = o.precision == SSA_PREC_F32C ? 0.0 : o.reorth_skip;
  cx.tol = o.tol > 0 ? o.tol : (o.precision == SSA_PREC_F32C ? 1e-7 * std::sqrt((double)lgMmax) : 1e-12);
  cx.max_restarts = o.max_restarts;
  cx.seed = o.seed;
  b->info.assign(4 * (size_t)nseries, 0);
#undef BCK2
  *out = b;
  return SSA_OK;
}

// Enqueue one run on the batch's stream: queue counters, slots, the
// persistent kernel (and the refinement).  Stream-ordered work only -- no
// allocation, host copy or synchronisation -- so a CUDA graph can capture it.
static int batch_enqueue(ssa_batch_t b, const double* fdev) {
  cudaStream_t s = b->stream;
  b->cx.f = fdev;
  BCK(cudaMemsetAsync(b->dnext, 0, 2 * sizeof(int), s));
  BCK(cudaMemsetAsync(b->slots, 0, (size_t)b->nslots * b->cx.slot_bytes, s));
  prof_begin(s);
  if (b->precision == SSA_PREC_F32C) k_batch_ssa<float, 16384><<<b->nslots, BT, B_SMEM, s>>>(b->cx);
  else k_batch_ssa<df64, 8192><<<b->nslots, BT, B_SMEM, s>>>(b->cx);
  prof_end(s, K_BATCH, 0.0, 0.0);
  BCK(cudaGetLastError());
  if (b->refine) {
    BRefine rf{b->dtw64, b->dA64, b->dB64, b->dnext + 1};
    prof_begin(s);
    k_batch_refine<<<b->nslots, BT, B_SMEM, s>>>(b->cx, rf);
    prof_end(s, K_BATCH, 0.0, 0.0);
    BCK(cudaGetLastError());
  }
  return SSA_OK;
}

// Wait for the last run and read the per-series status.
static int batch_finish(ssa_batch_t b) {
  cudaStream_t s = b->stream;
  BCK(cudaMemcpyAsync(b->info.data(), b->dinfo, b->info.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  int worst = SSA_OK;
  for (int i = 0; i < b->nseries; ++i) {
    const unsigned st = (unsigned)b->info[4 * i + 3];
    if (st & SSA_DEV_NONFINITE) worst = SSA_ENUMERIC;
    else if (!b->info[4 * i] && worst == SSA_OK) worst = SSA_ENOCONV;
  }
  if (worst == SSA_ENUMERIC) host_set_error("non-finite value in a batched series");
  if (worst == SSA_ENOCONV) host_set_error("a batched series did not converge within max_restarts");
  return worst;
}

// series data for a run: device pointers are used in place; host data is
// copied into the batch's own device buffer (pinned host memory keeps the
// copy capturable)
static int batch_input(ssa_batch_t b, const double* f, const double** fdev) {
  if (b_on_device(f)) {
    *fdev = f;
    return SSA_OK;
  }
  if (!b->fbuf) BCK(cudaMallocAsync(reinterpret_cast<void**>(&b->fbuf), std::max<int64_t>(b->ftot, 1) * sizeof(double),
                                    b->stream));
  BCK(cudaMemcpyAsync(b->fbuf, f, b->ftot * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  *fdev = b->fbuf;
  return SSA_OK;
}

extern "C" int ssa_decompose_batch(int nseries, const double* f, const int64_t* offsets, const int64_t* Ls,
                                   const int32_t* ks, const ssa_opts_t* opts, ssa_batch_t* out) {
  if (!f) return bfail(SSA_EINVAL, "f is NULL");
  int rc = batch_build(nseries, offsets, Ls, ks, opts, out);
  if (rc) return rc;
  ssa_batch_t b = *out;
  const double* fdev = nullptr;
  rc = batch_input(b, f, &fdev);
  if (!rc) rc = batch_enqueue(b, fdev);
  if (rc) {
    ssa_batch_destroy(b);
    *out = nullptr;
    return rc;
  }
  return batch_finish(b);
}

extern "C" int ssa_batch_plan(int nseries, const int64_t* offsets, const int64_t* Ls, const int32_t* ks,
                              const ssa_opts_t* opts, ssa_batch_t* out) {
  return batch_build(nseries, offsets, Ls, ks, opts, out);
}

extern "C" int ssa_batch_run(ssa_batch_t b, const double* f) {
  if (!b || !f) return bfail(SSA_EINVAL, "NULL argument");
  const double* fdev = nullptr;
  int rc = batch_input(b, f, &fdev);
  if (rc) return rc;
  return batch_enqueue(b, fdev);
}

extern "C" int ssa_batch_wait(ssa_batch_t b) {
  if (!b) return bfail(SSA_EINVAL, "NULL argument");
  return batch_finish(b);
}

namespace ssa {
const double* batch_device_U(ssa_batch_t b) { return b ? b->U : nullptr; }
}  // namespace ssa

extern "C" int ssa_batch_reconstruct(ssa_batch_t b, const int32_t* grp_off, const int32_t* grp_idx, int m,
                                     double* out) {
  if (!b || !grp_off || !grp_idx || !out || m < 1) return bfail(SSA_EINVAL, "NULL argument or m < 1");
  std::vector<int32_t> off, idx;
  int rc = to_host(grp_off, (size_t)m + 1, off);
  if (rc) return rc;
  if (off[0] != 0 || off[m] < 0) return bfail(SSA_EINVAL, "bad group offsets");
  rc = to_host(grp_idx, (size_t)std::max(off[m], 1), idx);
  if (rc) return rc;
  int kmin = 1 << 30;
  for (const BSeries& S : b->ser) kmin = std::min(kmin, S.k);
  std::vector<char> seen(kmin, 0);
  for (int gi = 0; gi < m; ++gi) {
    if (off[gi + 1] < off[gi]) return bfail(SSA_EINVAL, "bad group offsets");
    for (int a = off[gi]; a < off[gi + 1]; ++a) {
      if (idx[a] < 0 || idx[a] >= kmin) return bfail(SSA_EINVAL, "group index out of range for some series");
      if (seen[idx[a]]) return bfail(SSA_EINVAL, "groups overlap");
      seen[idx[a]] = 1;
    }
  }
  cudaStream_t s = b->stream;
  const int n = b->nseries;
  std::vector<int64_t> oo(n);
  int64_t tot = 0;
  int nmax = 2;
  for (int i = 0; i < n; ++i) {
    oo[i] = tot;
    tot += (int64_t)m * b->ser[i].N;
    nmax = std::max(nmax, 1 << b->ser[i].lg_n);
  }
  const int lgMmax = b->lg_Mmax;
  const int64_t Mmax = (int64_t)1 << lgMmax;
  const int lg_P = lgMmax - 1;
  const int64_t P = (int64_t)1 << lg_P;
  const int tws = (lgMmax + 1) / 2;
  const int64_t nA = Mmax >> tws, nB = (int64_t)1 << tws;
  std::vector<cplx<df64>> htw(P), hA(nA), hB(nB);
  for (int64_t q = 0; q < P; ++q) htw[q] = b_tw(q, P);
  for (int64_t q = 0; q < nA; ++q) hA[q] = b_tw(q << tws, Mmax);
  for (int64_t q = 0; q < nB; ++q) hB[q] = b_tw(q, Mmax);
  int dev = 0, sms = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int items = n * m;
  const int nblk = std::min(sms, items);
  const int64_t ld_scr = 2 * ((int64_t)nmax + 1);
  struct Bufs {
    cudaStream_t s;
    void* p[8] = {nullptr};
    ~Bufs() {
      for (void* q : p)
        if (q) cudaFreeAsync(q, s);
    }
  } bf{s};
  BCK(cudaMallocAsync(&bf.p[0], P * sizeof(cplx<df64>), s));
  BCK(cudaMallocAsync(&bf.p[1], nA * sizeof(cplx<df64>), s));
  BCK(cudaMallocAsync(&bf.p[2], nB * sizeof(cplx<df64>), s));
  BCK(cudaMallocAsync(&bf.p[3], (size_t)nblk * ld_scr * sizeof(cplx<df64>), s));
  BCK(cudaMallocAsync(&bf.p[4], (m + 1 + off[m] + 1) * sizeof(int), s));
  BCK(cudaMallocAsync(&bf.p[5], n * sizeof(int64_t) + n * sizeof(BSeries) + 16, s));
  BCK(cudaMallocAsync(&bf.p[6], sizeof(int), s));
  const bool odev = b_on_device(out);
  if (!odev) BCK(cudaMallocAsync(&bf.p[7], tot * sizeof(double), s));
  int* dgrp = static_cast<int*>(bf.p[4]);
  int64_t* doo = static_cast<int64_t*>(bf.p[5]);
  BSeries* dser = reinterpret_cast<BSeries*>(doo + n);
  BCK(cudaMemcpyAsync(bf.p[0], htw.data(), P * sizeof(cplx<df64>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(bf.p[1], hA.data(), nA * sizeof(cplx<df64>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(bf.p[2], hB.data(), nB * sizeof(cplx<df64>), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(dgrp, off.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(dgrp + m + 1, idx.data(), std::max(off[m], 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(doo, oo.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(dser, b->ser.data(), n * sizeof(BSeries), cudaMemcpyHostToDevice, s));
  BCK(cudaMemsetAsync(bf.p[6], 0, sizeof(int), s));
  BHCtx cx{};
  cx.ser = dser;
  cx.nseries = n;
  cx.m = m;
  cx.U = b->U;
  cx.V = b->V;
  cx.sigma = b->sigma;
  cx.grp_off = dgrp;
  cx.grp_idx = dgrp + m + 1;
  cx.out = odev ? out : static_cast<double*>(bf.p[7]);
  cx.out_off = doo;
  cx.tw = static_cast<cplx<df64>*>(bf.p[0]);
  cx.lg_P = lg_P;
  cx.tA = static_cast<cplx<df64>*>(bf.p[1]);
  cx.tB = static_cast<cplx<df64>*>(bf.p[2]);
  cx.tws = tws;
  cx.lg_Mmax = lgMmax;
  cx.scratch = static_cast<cplx<df64>*>(bf.p[3]);
  cx.ld_scr = ld_scr;
  cx.next = static_cast<int*>(bf.p[6]);
  prof_begin(s);
  if (b->precision == SSA_PREC_F32C) {
    auto kern = k_batch_hankel<float, 16384>;
    BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM));
    kern<<<nblk, BT, B_SMEM, s>>>(cx);
  } else {
    auto kern = k_batch_hankel<df64, 8192>;
    BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM));
    kern<<<nblk, BT, B_SMEM, s>>>(cx);
  }
  prof_end(s, K_HANKEL_SMALL, 8.0 * (double)(b->totU + b->totV) + 8.0 * (double)tot, 0.0);
  BCK(cudaGetLastError());
  if (!odev) BCK(cudaMemcpyAsync(out, bf.p[7], tot * sizeof(double), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  return SSA_OK;
}

extern "C" int ssa_batch_info(ssa_batch_t b, int i, int* k, int* converged, int* restarts, int64_t* matvecs) {
  if (!b || i < 0 || i >= b->nseries) return bfail(SSA_EINVAL, "bad batch handle or index");
  if (k) *k = b->ser[i].k;
  if (converged) *converged = b->info[4 * i];
  if (restarts) *restarts = b->info[4 * i + 1];
  if (matvecs) *matvecs = b->info[4 * i + 2];
  return SSA_OK;
}

extern "C" int ssa_batch_get(ssa_batch_t b, int i, double* sigma, double* U, double* V, double* resid) {
  if (!b || i < 0 || i >= b->nseries) return bfail(SSA_EINVAL, "bad batch handle or index");
  const BSeries& S = b->ser[i];
  cudaStream_t s = b->stream;
  if (sigma) BCK(cudaMemcpyAsync(sigma, b->sigma + S.out_s, S.k * sizeof(double), cudaMemcpyDefault, s));
  if (resid) BCK(cudaMemcpyAsync(resid, b->resid + S.out_s, S.k * sizeof(double), cudaMemcpyDefault, s));
  if (U) BCK(cudaMemcpyAsync(U, b->U + S.out_u, (size_t)S.L * S.k * sizeof(double), cudaMemcpyDefault, s));
  if (V) BCK(cudaMemcpyAsync(V, b->V + S.out_v, (size_t)S.K * S.k * sizeof(double), cudaMemcpyDefault, s));
  BCK(cudaStreamSynchronize(s));
  return SSA_OK;
}

extern "C" void ssa_batch_destroy(ssa_batch_t b) {
  if (!b) return;
  void* bufs[] = {b->U, b->V, b->sigma, b->resid, b->dtw, b->dA, b->dB, b->dtw64, b->dA64, b->dB64,
                  b->dser, b->dorder, b->dnext, b->dinfo, b->slots, b->fbuf};
  for (void* ptr : bufs)
    if (ptr) cudaFreeAsync(ptr, b->stream);
  delete b;
}
