// FFT-based trajectory-matrix products (Algorithms 2 and 3), the cached
// spectrum of the series (Algorithm 2 steps 1-2) and grouped rank-1
// Hankelization (Algorithm 4), for one CTA per transform (M <= 16384 in
// double-float, M <= 32768 in FP32) or a four-step decomposition over three
// kernels for large M.
//
// Index conventions (0-based; the series f[0..N-1] is the paper's f_1..f_N):
//   M >= N is the FFT length (a power of two), n = M/2 complex points.
//   c_j = f[N-L+j] for j < L, 0 for L <= j < L+M-N, f[j-L-(M-N)] beyond
//   (Algorithm 2 step 1 with M-N zeros between its two blocks, so every
//   M >= N embeds the same Toeplitz matrix);
//   X v  : w_j = v[K-1-j] (j < K), output p_0..p_{L-1}       (Algorithm 2)
//   X^T u: w_j = u[M-1-j] (j >= M-L), output p_{M-K}..p_{M-1} (Algorithm 3,
//          the printed slice p'_{L-1}..p'_N has one entry too many).
//   Hankelization: u' = (u, 0...), v' = (v, 0...) of length M >= L+K-1, the
//   linear convolution by FFT, divided by the antidiagonal counts
//   min(t+1, L, K, N-t) (Algorithm 4 prints a product with the counts; the
//   convolution identity of section 5 requires the quotient).
#include <cstdio>
#include <algorithm>
#include <vector>
#include <atomic>
#include <mutex>
#include "spectral.h"
#include "fft.cuh"
#include "prof.h"
#include "bulk.cuh"

namespace ssa {

// ---------------------------------------------------------------- loaders
template <class T> SSA_D T ld(const df64* p, int64_t i) { return scal<T>::from_df(p[i]); }
template <class T> SSA_D T ld(const double* p, int64_t i) { return scal<T>::from_double(__ldg(p + i)); }
SSA_D void st(df64* p, int64_t i, float v) { p[i] = make_df(v, 0.f); }
SSA_D void st(df64* p, int64_t i, df64 v) { p[i] = v; }
SSA_D void st(double* p, int64_t i, float v) { p[i] = (double)v; }
SSA_D void st(double* p, int64_t i, df64 v) { p[i] = df_to_double(v); }
SSA_D void st(double* p, int64_t i, double v) { p[i] = v; }
SSA_D void st(df64* p, int64_t i, double v) { p[i] = df_from_double(v); }
SSA_D double to_d(float v) { return (double)v; }
SSA_D double to_d(df64 v) { return df_to_double(v); }
SSA_D double to_d(double v) { return v; }
// Hankelization output: the value times os, a power of two that brings
// results computed with sigma scaled into range back to the caller's units
template <class V> SSA_D void st_os(double* p, int64_t i, V v, double os) { p[i] = to_d(v) * os; }
template <class V> SSA_D void st_os(df64* p, int64_t i, V v, double os) { st(p, i, to_d(v) * os); }

template <class T, int G, class In>
SSA_D T gather(const Geom& g, const In* x, int64_t glen, int64_t j) {
  if (G == GATHER_X) return j < g.K ? ld<T>(x, g.K - 1 - j) : scal<T>::zero();
  if (G == GATHER_XT) return j >= g.M - g.L ? ld<T>(x, g.M - 1 - j) : scal<T>::zero();
  if (G == GATHER_CIRC) {
    if (j < g.L) return ld<T>(x, g.N - g.L + j);
    const int64_t j0 = g.L + (g.M - g.N);
    return j >= j0 ? ld<T>(x, j - j0) : scal<T>::zero();
  }
  return j < glen ? ld<T>(x, j) : scal<T>::zero();  // GATHER_PAD
}

template <class T> SSA_D cplx<T> c_one() { return mk(scal<T>::from_double(1.0), scal<T>::zero()); }
// value of the arithmetic type T stored into a table of type tab_t<T>
template <class T> SSA_D tab_t<T> to_tab(cplx<T> v) {
  if constexpr (std::is_same<T, double>::value) return v;
  else return mk(scal<T>::to_df(v.re), scal<T>::to_df(v.im));
}
template <class T> SSA_D cplx<T> from_tab(tab_t<T> v) {
  if constexpr (std::is_same<T, double>::value) return v;
  else return mk(scal<T>::from_df(v.re), scal<T>::from_df(v.im));
}
// o += q, accumulated in the table's precision
template <class T> SSA_D void tab_acc(tab_t<T>& o, cplx<T> q) {
  if constexpr (std::is_same<T, double>::value) o = c_add(o, q);
  else o = mk(df_add(o.re, scal<T>::to_df(q.re)), df_add(o.im, scal<T>::to_df(q.im)));
}

SSA_D float cnt_recip_f(const Geom& g, int64_t t) {
  int64_t c = t + 1;
  if (g.N - t < c) c = g.N - t;
  const int64_t mn = g.L < g.K ? g.L : g.K;
  if (mn < c) c = mn;
  return (float)c;
}
template <class T> SSA_D T div_count(T v, float cnt);
template <> SSA_D float div_count<float>(float v, float cnt) { return v / cnt; }
template <> SSA_D df64 div_count<df64>(df64 v, float cnt) { return df_div(v, make_df(cnt, 0.f)); }
template <> SSA_D double div_count<double>(double v, float cnt) { return v / (double)cnt; }
template <class T> SSA_D T mul_scalar(T v, float s);
template <> SSA_D float mul_scalar<float>(float v, float s) { return v * s; }
template <> SSA_D df64 mul_scalar<df64>(df64 v, float s) { return df_mul_f(v, s); }
template <> SSA_D double mul_scalar<double>(double v, float s) { return v * (double)s; }

// ------------------------------------------------ single-CTA kernels
// Fused X v / X^T u: gather -> FFT -> real post-process -> x c-hat ->
// inverse pre-process -> inverse FFT -> window slice.  One CTA per vector.
template <class T, int THREADS, int MAXE, int G, class In, class Out>
__global__ void __launch_bounds__(THREADS) k_matvec_small(Geom g, const In* __restrict__ x, int64_t ldx,
                                                          Out* __restrict__ y, int64_t ldy,
                                                          const tab_t<T>* __restrict__ chat,
                                                          int64_t out_off, int64_t out_cnt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int n = 1 << g.lg_n;
  x += (int64_t)blockIdx.x * ldx;
  y += (int64_t)blockIdx.x * ldy;
  for (int t = threadIdx.x; t < n; t += THREADS)
    buf[t] = mk(gather<T, G>(g, x, 0, 2 * (int64_t)t), gather<T, G>(g, x, 0, 2 * (int64_t)t + 1));
  __syncthreads();
  cta_fft<T, THREADS, MAXE, false>(buf, g.lg_n, 1, g_tw<T>(g), g.lg_P);
  for (int k = threadIdx.x; k <= n / 2; k += THREADS) {
    const int nk = (n - k) & (n - 1);
    cplx<T> tw = k ? twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, (int64_t)(k) << g.twshift) : c_one<T>();
    cplx<T> wk, wnk, zk, znk;
    rfft_post(buf[k], buf[nk], tw, wk, wnk);
    cplx<T> pk = mul_spec(wk, chat[k]);
    cplx<T> pnk = mul_spec(wnk, chat[n - k]);
    irfft_pre(pk, pnk, tw, zk, znk);
    buf[k] = zk;
    if (k != 0 && nk != k) buf[nk] = znk;
  }
  __syncthreads();
  cta_fft<T, THREADS, MAXE, true>(buf, g.lg_n, 1, g_tw<T>(g), g.lg_P);
  for (int64_t m = threadIdx.x; m < out_cnt; m += THREADS) {
    const int64_t i = out_off + m;
    const cplx<T> z = buf[i >> 1];
    st(y, m, (i & 1) ? z.im : z.re);
  }
}

// Half spectrum W_0..W_n of a real length-M input (natural order), times scale.
template <class T, int THREADS, int MAXE, int G, class In>
__global__ void __launch_bounds__(THREADS) k_rfft_small(Geom g, const In* __restrict__ x, int64_t ldx, int64_t glen,
                                                        tab_t<T>* __restrict__ out, int64_t ldo, float scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int n = 1 << g.lg_n;
  x += (int64_t)blockIdx.x * ldx;
  out += (int64_t)blockIdx.x * ldo;
  for (int t = threadIdx.x; t < n; t += THREADS)
    buf[t] = mk(gather<T, G>(g, x, glen, 2 * (int64_t)t), gather<T, G>(g, x, glen, 2 * (int64_t)t + 1));
  __syncthreads();
  cta_fft<T, THREADS, MAXE, false>(buf, g.lg_n, 1, g_tw<T>(g), g.lg_P);
  const float s = 0.5f * scale;
  for (int k = threadIdx.x; k <= n / 2; k += THREADS) {
    const int nk = (n - k) & (n - 1);
    cplx<T> tw = k ? twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, (int64_t)(k) << g.twshift) : c_one<T>();
    cplx<T> wk, wnk;
    rfft_post(buf[k], buf[nk], tw, wk, wnk);
    wk = c_scale(wk, s);
    wnk = c_scale(wnk, s);
    out[k] = to_tab<T>(wk);
    out[n - k] = to_tab<T>(wnk);
  }
}

// Grouped rank-1 Hankelization (Algorithm 4 summed over a group): one CTA per
// group; u'_i and v'_i are transformed together (two length-n FFTs), the
// products sigma_i U_k V_k accumulate in registers, then one inverse FFT and
// the division by the antidiagonal counts.
template <class T, int THREADS, int MAXE, class Out>
__global__ void __launch_bounds__(THREADS) k_hankel_small(Geom g, const df64* __restrict__ U, int64_t ldu,
                                                          const df64* __restrict__ V, int64_t ldv,
                                                          const double* __restrict__ sigma,
                                                          const int* __restrict__ grp_off,
                                                          const int* __restrict__ grp_idx,
                                                          Out* __restrict__ out, int64_t ldo, double oscale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* bu = reinterpret_cast<cplx<T>*>(smem_raw);
  const int n = 1 << g.lg_n;
  cplx<T>* bv = bu + n;
  constexpr int MAXK = (MAXE / 4 + 1 + THREADS - 1) / THREADS;
  cplx<T> acc_k[MAXK], acc_nk[MAXK];
#pragma unroll
  for (int q = 0; q < MAXK; ++q) {
    acc_k[q] = mk(scal<T>::zero(), scal<T>::zero());
    acc_nk[q] = acc_k[q];
  }
  const int grp = blockIdx.x;
  const int i0 = grp_off[grp], i1 = grp_off[grp + 1];
  out += (int64_t)grp * ldo;
  for (int ii = i0; ii < i1; ++ii) {
    const int comp = grp_idx[ii];
    const df64* u = U + (int64_t)comp * ldu;
    const df64* v = V + (int64_t)comp * ldv;
    for (int t = threadIdx.x; t < n; t += THREADS) {
      const int64_t j = 2 * (int64_t)t;
      bu[t] = mk(gather<T, GATHER_PAD>(g, u, g.L, j), gather<T, GATHER_PAD>(g, u, g.L, j + 1));
      bv[t] = mk(gather<T, GATHER_PAD>(g, v, g.K, j), gather<T, GATHER_PAD>(g, v, g.K, j + 1));
    }
    __syncthreads();
    cta_fft<T, THREADS, MAXE, false>(bu, g.lg_n, 2, g_tw<T>(g), g.lg_P);
    const T sg = scal<T>::from_double(sigma[comp]);
#pragma unroll
    for (int q = 0; q < MAXK; ++q) {
      const int k = threadIdx.x + q * THREADS;
      if (k <= n / 2) {
        const int nk = (n - k) & (n - 1);
        cplx<T> tw = k ? twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, (int64_t)(k) << g.twshift) : c_one<T>();
        cplx<T> uk, unk, vk, vnk;
        rfft_post(bu[k], bu[nk], tw, uk, unk);
        rfft_post(bv[k], bv[nk], tw, vk, vnk);
        cplx<T> pk = c_mul(uk, vk), pnk = c_mul(unk, vnk);
        acc_k[q] = c_add(acc_k[q], mk(s_mul(pk.re, sg), s_mul(pk.im, sg)));
        acc_nk[q] = c_add(acc_nk[q], mk(s_mul(pnk.re, sg), s_mul(pnk.im, sg)));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < MAXK; ++q) {
    const int k = threadIdx.x + q * THREADS;
    if (k <= n / 2) {
      const int nk = (n - k) & (n - 1);
      cplx<T> tw = k ? twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, (int64_t)(k) << g.twshift) : c_one<T>();
      cplx<T> zk, znk;
      irfft_pre(acc_k[q], acc_nk[q], tw, zk, znk);
      bu[k] = zk;
      if (k != 0 && nk != k) bu[nk] = znk;
    }
  }
  __syncthreads();
  cta_fft<T, THREADS, MAXE, true>(bu, g.lg_n, 1, g_tw<T>(g), g.lg_P);
  // acc holds 4 sigma U V; irfft_pre doubles it; inverse FFT scales by n
  const float scale = 1.0f / (8.0f * (float)n);
  for (int64_t t = threadIdx.x; t < g.N; t += THREADS) {
    const cplx<T> z = bu[t >> 1];
    T p = (t & 1) ? z.im : z.re;
    st_os(out, t, div_count<T>(mul_scalar<T>(p, scale), cnt_recip_f(g, t)), oscale);
  }
}

// ------------------------------------------------ four-step kernels
// View the packed input z_t (t < n) as n1 x n2 row-major, t = n2 a + b.
// A: column FFTs over a, twiddle W_n^{b c}, store Y[c][b].
//
// Column tiles: a CTA takes cb = 2^lg_cb columns, held column after column
// in shared memory with one padding element per column (ld = n1 + 1) so that
// the transposing loads and stores spread over the banks.  Every global load
// of a thread (the gathered inputs, then the four-step twiddles) is issued
// before any of them is used: the loops run over a compile-time number of
// elements per thread.  The column FFTs read W_{n1}^m from a copy in shared
// memory (every (n2/n1)-th entry of the plan's W_{n2} table).
template <class T> SSA_HD size_t col_smem_bytes(int lg_n1, int lg_cb) {
  const size_t data = (size_t)(1 << lg_cb) * ((1 << lg_n1) + 1) * sizeof(cplx<T>);
  return (data + 15) / 16 * 16 + (size_t)(1 << lg_n1) * sizeof(tab_t<T>);
}

template <class T>
SSA_D tab_t<T>* col_twiddles(unsigned char* smem, const Geom& g, int lg_cb, int threads) {
  const int n1 = 1 << g.lg_n1;
  const size_t data = (size_t)(1 << lg_cb) * (n1 + 1) * sizeof(cplx<T>);
  tab_t<T>* tws = reinterpret_cast<tab_t<T>*>(smem + (data + 15) / 16 * 16);
  const tab_t<T>* tw = g_tw<T>(g);
  for (int m = threadIdx.x; m < n1; m += threads) tws[m] = tw[(int64_t)m << (g.lg_P - g.lg_n1)];
  return tws;
}

// col_of_row (may be null): batch row y transforms column col_of_row[y] of x.
template <class T, int THREADS, int MAXE, int G, class In>
__global__ void __launch_bounds__(THREADS) k_fs_col_fwd(Geom g, const In* __restrict__ x, int64_t ldx, int64_t glen,
                                                        cplx<T>* __restrict__ Y, int lg_cb,
                                                        const int* __restrict__ col_of_row) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int cb = 1 << lg_cb, ld = (1 << g.lg_n1) + 1;
  const int b0 = blockIdx.x << lg_cb;
  const int64_t n = (int64_t)1 << g.lg_n;
  x += (int64_t)(col_of_row ? col_of_row[blockIdx.y] : (int)blockIdx.y) * ldx;
  Y += (int64_t)blockIdx.y * n;
  const int E = cb << g.lg_n1;
  constexpr int EPT = (MAXE + THREADS - 1) / THREADS;
  {
    cplx<T> v[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = threadIdx.x + q * THREADS;
      if (e < E) {
        const int bb = e & (cb - 1), a = e >> lg_cb;
        const int64_t t = ((int64_t)a << g.lg_n2) + b0 + bb;
        v[q] = mk(gather<T, G>(g, x, glen, 2 * t), gather<T, G>(g, x, glen, 2 * t + 1));
      }
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = threadIdx.x + q * THREADS;
      if (e < E) buf[(e & (cb - 1)) * ld + (e >> lg_cb)] = v[q];
    }
  }
  const tab_t<T>* tws = col_twiddles<T>(smem_raw, g, lg_cb, THREADS);
  __syncthreads();
  cta_fft_tw<T, THREADS, MAXE, false>(buf, g.lg_n1, cb, TwShared<T>{tws}, g.lg_n1, ld);
  cplx<T> tv[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = threadIdx.x + q * THREADS;
    if (e < E) {
      const int64_t b = b0 + (e & (cb - 1));
      const int c = e >> lg_cb;
      const int64_t m = 2 * ((b * c) & (n - 1));
      tv[q] = m ? twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, m << g.twshift) : c_one<T>();
    }
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = threadIdx.x + q * THREADS;
    if (e < E) {
      const int bb = e & (cb - 1), c = e >> lg_cb;
      const int64_t b = b0 + bb;
      cplx<T> v = buf[bb * ld + c];
      if (2 * ((b * c) & (n - 1))) v = c_mul(v, tv[q]);
      Y[((int64_t)c << g.lg_n2) + b] = v;
    }
  }
}

// B: row pass over rows c and n1-c (block 0: rows 0 and n1/2).
template <class T, int THREADS, int MAXE, int MODE>
__global__ void __launch_bounds__(THREADS) k_fs_row(Geom g, cplx<T>* __restrict__ Y, RowArgs ra) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int n1 = 1 << g.lg_n1, n2 = 1 << g.lg_n2;
  const int64_t n = (int64_t)1 << g.lg_n;
  const int r0 = blockIdx.x == 0 ? 0 : blockIdx.x;
  const int r1 = blockIdx.x == 0 ? n1 / 2 : n1 - blockIdx.x;
  Y += (int64_t)blockIdx.y * n;
  if (MODE != ROW_INV_LOAD) {
    for (int e = threadIdx.x; e < 2 * n2; e += THREADS) {
      const int row = e < n2 ? r0 : r1;
      buf[e] = Y[((int64_t)row << g.lg_n2) + (e & (n2 - 1))];
    }
    __syncthreads();
    cta_fft<T, THREADS, MAXE, false>(buf, g.lg_n2, 2, g_tw<T>(g), g.lg_P);
  }
  const int npairs = blockIdx.x == 0 ? n2 + 1 : n2;
  using TT = tab_t<T>;
  const TT* chat = static_cast<const TT*>(ra.chat);
  const TT* sin_ = ra.spec_in ? static_cast<const TT*>(ra.spec_in) + (int64_t)blockIdx.y * ra.ld_spec : nullptr;
  const int orow = (MODE == ROW_FWD_MUL_ACC && ra.out_of_row) ? ra.out_of_row[blockIdx.y] : (int)blockIdx.y;
  TT* sout = ra.spec_out ? static_cast<TT*>(ra.spec_out) + (int64_t)orow * ra.ld_spec : nullptr;
  for (int p = threadIdx.x; p < npairs; p += THREADS) {
    int sa, sb, ca, ea, cbr, eb;  // smem slots and (row, column) of the pair members
    if (blockIdx.x == 0) {
      if (p <= n2 / 2) {
        ca = 0; ea = p; cbr = 0; eb = (n2 - p) & (n2 - 1);
        sa = ea; sb = eb;
      } else {
        const int q = p - (n2 / 2 + 1);
        ca = n1 / 2; ea = q; cbr = n1 / 2; eb = n2 - 1 - q;
        sa = n2 + ea; sb = n2 + eb;
      }
    } else {
      ca = r0; ea = p; cbr = r1; eb = n2 - 1 - p;
      sa = ea; sb = n2 + eb;
    }
    const int64_t k = (int64_t)ca + ((int64_t)ea << g.lg_n1);   // natural index of member a
    const bool k0 = (k == 0);
    // perm-layout positions (row-major c * n2 + e); the partner of k = 0 is index n
    const int64_t pa = ((int64_t)ca << g.lg_n2) + ea;
    const int64_t pb = k0 ? n : ((int64_t)cbr << g.lg_n2) + eb;
    cplx<T> tw = k0 ? c_one<T>() : twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, (int64_t)(k) << g.twshift);
    cplx<T> pk, pnk;
    if (MODE == ROW_INV_LOAD) {
      pk = from_tab<T>(sin_[pa]);
      pnk = from_tab<T>(sin_[pb]);
    } else {
      cplx<T> wk, wnk;
      rfft_post(buf[sa], buf[sb], tw, wk, wnk);
      if (MODE == ROW_MATVEC) {
        pk = mul_spec(wk, chat[pa]);
        pnk = mul_spec(wnk, chat[pb]);
      } else if (MODE == ROW_FWD_STORE) {
        const float s = 0.5f * ra.scale;
        wk = c_scale(wk, s);
        wnk = c_scale(wnk, s);
        const int64_t oa = ra.natural ? k : pa;
        const int64_t ob = ra.natural ? (k0 ? n : n - k) : pb;
        sout[oa] = to_tab<T>(wk);
        if (!(k != 0 && sa == sb)) sout[ob] = to_tab<T>(wnk);
        continue;
      } else {  // ROW_FWD_MUL_ACC: spec_out += weight * spec_in * W
        const int wi = ra.weight_of_row ? ra.weight_of_row[blockIdx.y] : ra.weight_idx;
        const T sg = scal<T>::from_double(ra.weight[wi] * 0.5);
        cplx<T> qa = c_mul(from_tab<T>(sin_[pa]), wk), qb = c_mul(from_tab<T>(sin_[pb]), wnk);
        qa = mk(s_mul(qa.re, sg), s_mul(qa.im, sg));
        qb = mk(s_mul(qb.re, sg), s_mul(qb.im, sg));
        tab_acc<T>(sout[pa], qa);
        if (!(k != 0 && sa == sb)) tab_acc<T>(sout[pb], qb);
        continue;
      }
    }
    cplx<T> zk, znk;
    irfft_pre(pk, pnk, tw, zk, znk);
    buf[sa] = zk;
    if (!k0 && sb != sa) buf[sb] = znk;
  }
  if (MODE == ROW_FWD_STORE || MODE == ROW_FWD_MUL_ACC) return;
  __syncthreads();
  cta_fft<T, THREADS, MAXE, true>(buf, g.lg_n2, 2, g_tw<T>(g), g.lg_P);
  for (int e = threadIdx.x; e < 2 * n2; e += THREADS) {
    const int row = e < n2 ? r0 : r1;
    const int64_t b = e & (n2 - 1);
    cplx<T> v = buf[e];
    const int64_t m = 2 * ((b * row) & (n - 1));
    if (m) v = c_mul_conj(v, twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, (int64_t)(m) << g.twshift));
    Y[((int64_t)row << g.lg_n2) + b] = v;
  }
}

// Set (never cleared by the kernels) when a bounded wait of a spectral kernel
// ran out; read with spectral_fault_read.
__device__ unsigned g_spectral_fault;
constexpr unsigned BULK_WAIT_LIMIT = 1u << 24;

// B for the products (ROW_MATVEC), rows staged by TMA bulk copies: one
// thread arms an mbarrier and copies rows r0 and r1 of Y, the same two rows
// of the spectrum (four-step order, row c at c * n2), the twiddle table
// W_{n2}^m and the first n2/2 entries of the two-level table tA into shared
// memory, all in flight at once.  The row FFTs then read their twiddles from
// shared memory, and the real-FFT post-processing takes W_M^k, k = c + e n1,
// as tA[e >> 1] tB[c + (e & 1) n1] (the two-level split at tws = lg_n1 + 1),
// the same operands as twiddle_M.  The inverse four-step twiddles are
// gathered from the global tables with all loads of a thread issued before
// use.  Requires lg_P == lg_n2 (four-step plans).  Arithmetic and operands are
// those of k_fs_row<T, ..., ROW_MATVEC>, so the results are the same bit for bit.
template <class T, int THREADS, int MAXE>
__global__ void __launch_bounds__(THREADS) k_fs_row_mv(Geom g, cplx<T>* __restrict__ Y,
                                                       const cplx<df64>* __restrict__ chat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ cplx<df64> tbs[4];   // tB[c], tB[c + n1] for the two rows
  __shared__ cplx<df64> chat_n;   // C_n, the partner of k = 0 (block 0)
  const int n1 = 1 << g.lg_n1, n2 = 1 << g.lg_n2;
  const int64_t n = (int64_t)1 << g.lg_n;
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);                  // rows r0 | r1 of Y
  cplx<df64>* cs = reinterpret_cast<cplx<df64>*>(buf + 2 * n2);          // rows r0 | r1 of the spectrum
  cplx<df64>* tws = cs + 2 * n2;                                          // W_{n2}^m, m < n2
  cplx<df64>* tas = tws + n2;                                             // tA[0 .. n2/2)
  const int r0 = blockIdx.x;
  const int r1 = blockIdx.x == 0 ? n1 / 2 : n1 - blockIdx.x;
  Y += (int64_t)blockIdx.y * n;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    const unsigned yb = (unsigned)(n2 * sizeof(cplx<T>)), cb = (unsigned)(n2 * sizeof(cplx<df64>));
    mbar_expect_tx(&bar, 2 * yb + 2 * cb + cb + cb / 2);
    bulk_g2s(buf, Y + ((int64_t)r0 << g.lg_n2), yb, &bar);
    bulk_g2s(buf + n2, Y + ((int64_t)r1 << g.lg_n2), yb, &bar);
    bulk_g2s(cs, chat + ((int64_t)r0 << g.lg_n2), cb, &bar);
    bulk_g2s(cs + n2, chat + ((int64_t)r1 << g.lg_n2), cb, &bar);
    bulk_g2s(tws, g.tw, cb, &bar);
    bulk_g2s(tas, g.tA, cb / 2, &bar);
  }
  if (threadIdx.x < 4) {
    const int c = threadIdx.x < 2 ? r0 : r1;
    tbs[threadIdx.x] = g.tB[c + (threadIdx.x & 1) * n1];
  }
  if (threadIdx.x == 4) chat_n = chat[n];
  __syncthreads();  // the barrier is initialised before anyone polls it
  if (!mbar_wait(&bar, 0, BULK_WAIT_LIMIT)) {
    atomicOr(&g_spectral_fault, 1u);
    mbar_wait(&bar, 0, BULK_WAIT_LIMIT);  // give the copies in flight one more bounded wait
    return;
  }
  const TwShared<T> twsm{tws};
  cta_fft_tw<T, THREADS, MAXE, false>(buf, g.lg_n2, 2, twsm, g.lg_P);
  const int npairs = blockIdx.x == 0 ? n2 + 1 : n2;
  for (int p = threadIdx.x; p < npairs; p += THREADS) {
    int sa, sb, ca, ea;  // smem slots of the pair members, (row, column) of member a
    int ra;              // 0: member a in row r0 (block 0: row 0), 1: row r1
    if (blockIdx.x == 0) {
      if (p <= n2 / 2) {
        ca = 0; ea = p; ra = 0;
        sa = ea; sb = (n2 - p) & (n2 - 1);
      } else {
        const int q = p - (n2 / 2 + 1);
        ca = n1 / 2; ea = q; ra = 1;
        sa = n2 + ea; sb = n2 + (n2 - 1 - q);
      }
    } else {
      ca = r0; ea = p; ra = 0;
      sa = ea; sb = n2 + (n2 - 1 - p);
    }
    const bool k0 = (ca == 0 && ea == 0);
    // W_M^k, k = ca + ea n1, from the two-level table (tA[k >> tws] tB[k & mask])
    const cplx<T> tw = k0 ? c_one<T>() : c_mul(from_tab<T>(tas[ea >> 1]), from_tab<T>(tbs[2 * ra + (ea & 1)]));
    cplx<T> wk, wnk;
    rfft_post(buf[sa], buf[sb], tw, wk, wnk);
    const cplx<T> pk = mul_spec(wk, cs[sa]);
    const cplx<T> pnk = mul_spec(wnk, k0 ? chat_n : cs[sb]);
    cplx<T> zk, znk;
    irfft_pre(pk, pnk, tw, zk, znk);
    buf[sa] = zk;
    if (!k0 && sb != sa) buf[sb] = znk;
  }
  __syncthreads();
  cta_fft_tw<T, THREADS, MAXE, true>(buf, g.lg_n2, 2, twsm, g.lg_P);
  // conj(W_n^{b row}) on the way out, all table loads of this thread first
  constexpr int EPT = (MAXE + THREADS - 1) / THREADS;
  cplx<T> tv[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = threadIdx.x + q * THREADS;
    if (e < 2 * n2) {
      const int row = e < n2 ? r0 : r1;
      const int64_t b = e & (n2 - 1);
      const int64_t m = 2 * ((b * row) & (n - 1));
      tv[q] = m ? twiddle_M<T>(g_tA<T>(g), g_tB<T>(g), g.tws, m << g.twshift) : c_one<T>();
    }
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = threadIdx.x + q * THREADS;
    if (e < 2 * n2) {
      const int row = e < n2 ? r0 : r1;
      const int64_t b = e & (n2 - 1);
      const int64_t m = 2 * ((b * row) & (n - 1));
      cplx<T> v = buf[e];
      if (m) v = c_mul_conj(v, tv[q]);
      Y[((int64_t)row << g.lg_n2) + b] = v;
    }
  }
}

int spectral_fault_read(unsigned* host, cudaStream_t s) {
  return (int)cudaMemcpyFromSymbolAsync(host, g_spectral_fault, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
}

// C: inverse column FFTs over c, unpack the real output and write the slice
// (matvec) or the count-divided series (Hankelization).
template <class T, int THREADS, int MAXE, int OUTM, class Out>
__global__ void __launch_bounds__(THREADS) k_fs_col_inv(Geom g, const cplx<T>* __restrict__ Y, Out* __restrict__ y,
                                                        int64_t ldy, int64_t out_off, int64_t out_cnt, float scale,
                                                        int lg_cb, double oscale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int cb = 1 << lg_cb, ld = (1 << g.lg_n1) + 1;  // padded column tile, as in k_fs_col_fwd
  const int b0 = blockIdx.x << lg_cb;
  const int64_t n = (int64_t)1 << g.lg_n;
  Y += (int64_t)blockIdx.y * n;
  y += (int64_t)blockIdx.y * ldy;
  const int E = cb << g.lg_n1;
  constexpr int EPT = (MAXE + THREADS - 1) / THREADS;
  {
    cplx<T> v[EPT];  // all loads of this thread in flight before the first store
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = threadIdx.x + q * THREADS;
      if (e < E) v[q] = Y[((int64_t)(e >> lg_cb) << g.lg_n2) + b0 + (e & (cb - 1))];
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = threadIdx.x + q * THREADS;
      if (e < E) buf[(e & (cb - 1)) * ld + (e >> lg_cb)] = v[q];
    }
  }
  const tab_t<T>* tws = col_twiddles<T>(smem_raw, g, lg_cb, THREADS);
  __syncthreads();
  cta_fft_tw<T, THREADS, MAXE, true>(buf, g.lg_n1, cb, TwShared<T>{tws}, g.lg_n1, ld);
#pragma unroll
  for (int q = 0; q < 2 * EPT; ++q) {
    const int e = threadIdx.x + q * THREADS;
    if (e >= 2 * E) break;
    const int half = e & 1;
    const int ee = e >> 1;
    const int bb = ee & (cb - 1), a = ee >> lg_cb;
    const int64_t t = ((int64_t)a << g.lg_n2) + b0 + bb;
    const int64_t i = 2 * t + half;
    const cplx<T> z = buf[bb * ld + a];
    T v = half ? z.im : z.re;
    if (OUTM == OUT_SLICE) {
      if (i >= out_off && i < out_off + out_cnt) st(y, i - out_off, mul_scalar<T>(v, scale));
    } else {
      if (i < g.N) st_os(y, i, div_count<T>(mul_scalar<T>(v, scale), cnt_recip_f(g, i)), oscale);
    }
  }
}

// ------------------------------------------------ host launchers
static int lg2(int64_t x) {
  int r = 0;
  while (((int64_t)1 << r) < x) ++r;
  return r;
}

// MAXE: largest single-CTA transform (128 KB of shared memory, 512 threads);
// COLE: elements per CTA of the four-step column kernels (32 KB, 256 threads),
// small enough for several CTAs per SM and no register spills.
template <class T> struct Lim;
template <> struct Lim<float> { static constexpr int MAXE = SMALL_MAXE_F32; static constexpr int COLE = 4096; };
template <> struct Lim<df64> { static constexpr int MAXE = SMALL_MAXE_DF64; static constexpr int COLE = 2048; };
template <> struct Lim<double> { static constexpr int MAXE = SMALL_MAXE_DF64; static constexpr int COLE = 2048; };
constexpr int TH = 512;
constexpr int TH_ROW = 256;
constexpr int MAXE_ROW = 4096;

// Opt each kernel into the dynamic shared memory it needs, once per size
// (fixed table, no heap allocation).
template <class K> static void set_smem(K kern, size_t bytes) {
  static std::mutex mu;
  static const void* keys[128];
  static size_t vals[128];
  static int used = 0;
  if (bytes <= 48 * 1024) return;
  std::lock_guard<std::mutex> lock(mu);
  const void* key = reinterpret_cast<const void*>(kern);
  int i = 0;
  while (i < used && keys[i] != key) ++i;
  if (i == used) {
    if (used == 128) {  // table full: set the attribute every time
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      return;
    }
    keys[used] = key;
    vals[used] = 0;
    ++used;
  }
  if (bytes > vals[i]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    vals[i] = bytes;
  }
}

bool small_path(const Geom& g, int prec) {
  const int lim = prec == PREC_F32C ? Lim<float>::MAXE : Lim<df64>::MAXE;
  return ((int64_t)1 << g.lg_n) <= lim;
}

int col_lg_cb(const Geom& g, int maxe) {
  int lg = lg2(maxe) - g.lg_n1;
  if (lg > g.lg_n2) lg = g.lg_n2;
  if (lg < 0) lg = 0;
  return lg;
}

// Columns per CTA (2^lg_cb) and threads per CTA of the four-step column
// passes, and threads per CTA of the row pass.  Every choice gives bitwise the
// same result (each butterfly computes the same operations whichever thread
// runs it); autotune_fourstep() times the candidates once per (arithmetic
// type, pass, n) and the launches below use the fastest, else the largest
// tile with 256 threads.  A tuned column entry holds lg_cb | (thread index << 8),
// thread index 0, 1, 2 for 128, 256, 512 threads; a row entry 0, 1 for 256, 512.
template <class T> constexpr int type_slot() { return std::is_same<T, float>::value ? 0 : 1; }
static std::atomic<int> g_tuned_cb[2][2][32];
static std::atomic<int> g_tuned_row[2][32];
constexpr int COL_THREADS[3] = {128, 256, 512};
static std::atomic<bool> g_tune_init{false};
static std::mutex g_tune_mu;
static void tune_table_init() {
  if (g_tune_init.load()) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune_init.load()) return;
  for (auto& a : g_tuned_cb)
    for (auto& b : a)
      for (auto& c : b) c.store(-1);
  for (auto& a : g_tuned_row)
    for (auto& b : a) b.store(-1);
  g_tune_init.store(true);
}
// tuned column tile: lg_cb | (thread index << 8)
template <class T> static int tuned_col(const Geom& g, int pass) {
  const int dflt = col_lg_cb(g, Lim<T>::COLE) | (1 << 8);
  if (std::is_same<T, double>::value || !g_tune_init.load()) return dflt;
  const int v = g_tuned_cb[type_slot<T>()][pass][g.lg_n].load();
  return v >= 0 && (v & 0xff) <= (dflt & 0xff) ? v : dflt;
}
template <class T> static int tuned_row_threads(const Geom& g) {
  if (std::is_same<T, double>::value || !g_tune_init.load()) return 256;
  return g_tuned_row[type_slot<T>()][g.lg_n].load() == 1 ? 512 : 256;
}

template <class T, int G, class In, int TH>
static void fs_forward_th(const Geom& g, const In* x, int64_t ldx, int64_t glen, cplx<T>* Y, int batch, cudaStream_t s,
                          int lg_cb, const int* col_of_row) {
  constexpr int MAXE = Lim<T>::COLE;
  const size_t sm = col_smem_bytes<T>(g.lg_n1, lg_cb);
  auto kern = k_fs_col_fwd<T, TH, MAXE, G, In>;
  set_smem(kern, sm);
  dim3 grid((1 << g.lg_n2) >> lg_cb, batch);
  kern<<<grid, TH, sm, s>>>(g, x, ldx, glen, Y, lg_cb, col_of_row);
}
// tile: lg_cb | (thread index << 8); -1 = the tuned (or default) tile
template <class T, int G, class In>
static void fs_forward(const Geom& g, const In* x, int64_t ldx, int64_t glen, cplx<T>* Y, int batch, cudaStream_t s,
                       int cls, double bytes, int tile = -1, const int* col_of_row = nullptr) {
  const int v = tile >= 0 ? tile : tuned_col<T>(g, 0);
  const int lg_cb = v & 0xff, th = (v >> 8) & 3;
  prof_begin(s);
  if (th == 0) fs_forward_th<T, G, In, 128>(g, x, ldx, glen, Y, batch, s, lg_cb, col_of_row);
  else if (th == 2) fs_forward_th<T, G, In, 512>(g, x, ldx, glen, Y, batch, s, lg_cb, col_of_row);
  else fs_forward_th<T, G, In, 256>(g, x, ldx, glen, Y, batch, s, lg_cb, col_of_row);
  prof_end(s, cls, bytes, 5.0 * (double)((int64_t)1 << g.lg_n) * g.lg_n1 * batch, 1);
}

template <class T, int TH>
static void row_mv_th(const Geom& g, cplx<T>* Y, const cplx<df64>* chat, int batch, cudaStream_t s) {
  const size_t n2 = (size_t)1 << g.lg_n2;
  const size_t sm = 2 * n2 * sizeof(cplx<T>) + (2 * n2 + n2) * sizeof(cplx<df64>) + n2 / 2 * sizeof(cplx<df64>);
  auto kern = (2 << g.lg_n2) <= MAXE_ROW / 2 ? k_fs_row_mv<T, TH, MAXE_ROW / 2> : k_fs_row_mv<T, TH, MAXE_ROW>;
  set_smem(kern, sm);
  dim3 grid((1 << g.lg_n1) / 2, batch);
  kern<<<grid, TH, sm, s>>>(g, Y, chat);
}
// the staged row pass applies to four-step products whose buffers and tables
// start on 16-byte boundaries (bulk copies need them); otherwise k_fs_row runs
template <class T> static bool row_mv_applies(const Geom& g, const void* Y = nullptr, const void* chat = nullptr) {
  const uintptr_t al = reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(chat) |
                       reinterpret_cast<uintptr_t>(g.tw) | reinterpret_cast<uintptr_t>(g.tA);
  return !std::is_same<T, double>::value && g.lg_P == g.lg_n2 && g.twshift == 0 && (2 << g.lg_n2) <= MAXE_ROW &&
         (al & 15) == 0;
}

template <class T, int MODE>
static void fs_row(const Geom& g, cplx<T>* Y, const RowArgs& ra, int batch, cudaStream_t s, int cls, double bytes,
                   int threads = 0) {
  if constexpr (MODE == ROW_MATVEC && !std::is_same<T, double>::value) {
    if (row_mv_applies<T>(g, Y, ra.chat)) {
      const int th = threads > 0 ? threads : tuned_row_threads<T>(g);
      prof_begin(s);
      if (th == 512) row_mv_th<T, 512>(g, Y, static_cast<const cplx<df64>*>(ra.chat), batch, s);
      else row_mv_th<T, 256>(g, Y, static_cast<const cplx<df64>*>(ra.chat), batch, s);
      prof_end(s, cls, bytes, 10.0 * (double)((int64_t)1 << g.lg_n) * g.lg_n2 * batch, 1);
      return;
    }
  }
  const size_t sm = (size_t)(2 << g.lg_n2) * sizeof(cplx<T>);
  // the register arrays of the in-place FFT are sized by the bound: use the
  // smaller instantiation for rows of up to 1024 points
  auto kern = (2 << g.lg_n2) <= MAXE_ROW / 2 ? k_fs_row<T, TH_ROW, MAXE_ROW / 2, MODE>
                                             : k_fs_row<T, TH_ROW, MAXE_ROW, MODE>;
  set_smem(kern, sm);
  dim3 grid((1 << g.lg_n1) / 2, batch);
  prof_begin(s);
  kern<<<grid, TH_ROW, sm, s>>>(g, Y, ra);
  prof_end(s, cls, bytes, 10.0 * (double)((int64_t)1 << g.lg_n) * g.lg_n2 * batch, 1);
}

template <class T, int OUTM, class Out, int TH>
static void fs_inverse_th(const Geom& g, const cplx<T>* Y, Out* y, int64_t ldy, int64_t off, int64_t cnt, float scale,
                          int batch, cudaStream_t s, int lg_cb, double oscale) {
  constexpr int MAXE = Lim<T>::COLE;
  const size_t sm = col_smem_bytes<T>(g.lg_n1, lg_cb);
  auto kern = k_fs_col_inv<T, TH, MAXE, OUTM, Out>;
  set_smem(kern, sm);
  dim3 grid((1 << g.lg_n2) >> lg_cb, batch);
  kern<<<grid, TH, sm, s>>>(g, Y, y, ldy, off, cnt, scale, lg_cb, oscale);
}
template <class T, int OUTM, class Out>
static void fs_inverse(const Geom& g, const cplx<T>* Y, Out* y, int64_t ldy, int64_t off, int64_t cnt, float scale,
                       int batch, cudaStream_t s, int cls, double bytes, int tile = -1, double oscale = 1.0) {
  const int v = tile >= 0 ? tile : tuned_col<T>(g, 1);
  const int lg_cb = v & 0xff, th = (v >> 8) & 3;
  prof_begin(s);
  if (th == 0) fs_inverse_th<T, OUTM, Out, 128>(g, Y, y, ldy, off, cnt, scale, batch, s, lg_cb, oscale);
  else if (th == 2) fs_inverse_th<T, OUTM, Out, 512>(g, Y, y, ldy, off, cnt, scale, batch, s, lg_cb, oscale);
  else fs_inverse_th<T, OUTM, Out, 256>(g, Y, y, ldy, off, cnt, scale, batch, s, lg_cb, oscale);
  prof_end(s, cls, bytes, 5.0 * (double)((int64_t)1 << g.lg_n) * g.lg_n1 * batch, 1);
}

// ---- public launchers (spectral.h)

template <class T, class In, class Out>
static void matvec_impl(const Geom& g, int transpose, const In* x, int64_t ldx, Out* y, int64_t ldy, int batch,
                        const tab_t<T>* chat, void* scratch, bool small, cudaStream_t s) {
  const int64_t off = transpose ? g.M - g.K : 0;
  const int64_t cnt = transpose ? g.K : g.L;
  // algorithmic traffic of a product (section 8(d)): the input and output
  // vectors and the half spectrum; flops of two real FFTs and the multiply
  const double n = (double)((int64_t)1 << g.lg_n);
  const double in_b = (double)sizeof(In) * (transpose ? g.L : g.K) * batch;
  const double out_b = (double)sizeof(Out) * cnt * batch;
  const double spec_b = 16.0 * (n + 1);
  const double mv_bytes = in_b + out_b + spec_b;
  const double mv_flops = (5.0 * (double)g.M * (g.lg_n + 1) + 3.0 * (double)g.M) * batch;
  if (small) {
    constexpr int MAXE = Lim<T>::MAXE;
    const size_t sm = (size_t)(1 << g.lg_n) * sizeof(cplx<T>);
    if (transpose) {
      auto kern = k_matvec_small<T, TH, MAXE, GATHER_XT, In, Out>;
      set_smem(kern, sm);
      prof_begin(s);
      kern<<<batch, TH, sm, s>>>(g, x, ldx, y, ldy, chat, off, cnt);
      prof_end(s, K_MATVEC_SMALL, mv_bytes, mv_flops);
    } else {
      auto kern = k_matvec_small<T, TH, MAXE, GATHER_X, In, Out>;
      set_smem(kern, sm);
      prof_begin(s);
      kern<<<batch, TH, sm, s>>>(g, x, ldx, y, ldy, chat, off, cnt);
      prof_end(s, K_MATVEC_SMALL, mv_bytes, mv_flops);
    }
    return;
  }
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(scratch);
  if (transpose) fs_forward<T, GATHER_XT, In>(g, x, ldx, 0, Y, batch, s, K_MATVEC_COLFWD, in_b);
  else fs_forward<T, GATHER_X, In>(g, x, ldx, 0, Y, batch, s, K_MATVEC_COLFWD, in_b);
  RowArgs ra{};
  ra.chat = chat;
  fs_row<T, ROW_MATVEC>(g, Y, ra, batch, s, K_MATVEC_ROW, spec_b);
  fs_inverse<T, OUT_SLICE, Out>(g, Y, y, ldy, off, cnt, 1.0f, batch, s, K_MATVEC_COLINV, out_b);
}

void launch_matvec_df(const Geom& g, int prec, int transpose, const df64* x, int64_t ldx, df64* y, int64_t ldy,
                      int batch, const cplx<df64>* chat, void* scratch, cudaStream_t s) {
  const bool sm = small_path(g, prec);
  if (prec == PREC_F32C) matvec_impl<float, df64, df64>(g, transpose, x, ldx, y, ldy, batch, chat, scratch, sm, s);
  else matvec_impl<df64, df64, df64>(g, transpose, x, ldx, y, ldy, batch, chat, scratch, sm, s);
}

void launch_matvec_d(const Geom& g, int prec, int transpose, const double* x, int64_t ldx, double* y, int64_t ldy,
                     int batch, const cplx<df64>* chat, void* scratch, cudaStream_t s) {
  const bool sm = small_path(g, prec);
  if (prec == PREC_F32C) matvec_impl<float, double, double>(g, transpose, x, ldx, y, ldy, batch, chat, scratch, sm, s);
  else matvec_impl<df64, double, double>(g, transpose, x, ldx, y, ldy, batch, chat, scratch, sm, s);
}

bool native_small(const Geom& g) { return ((int64_t)1 << g.lg_n) <= Lim<double>::MAXE; }

void launch_matvec_native(const Geom& g, int transpose, const double* x, int64_t ldx, double* y, int64_t ldy,
                          int batch, const cplx<double>* chat, void* scratch, cudaStream_t s) {
  const bool sm = native_small(g);
  matvec_impl<double, double, double>(g, transpose, x, ldx, y, ldy, batch, chat, scratch, sm, s);
}

// Spectrum of the circulant column, always in df64.  natural: 1 -> index k,
// 0 -> four-step row-major order (c * n2 + e) with W_n at index n.
void launch_spectrum(const Geom& g, const double* f, cplx<df64>* chat, int natural, float scale, void* scratch,
                     cudaStream_t s) {
  if (((int64_t)1 << g.lg_n) <= Lim<df64>::MAXE) {
    const size_t sm = (size_t)(1 << g.lg_n) * sizeof(cplx<df64>);
    auto kern = k_rfft_small<df64, TH, Lim<df64>::MAXE, GATHER_CIRC, double>;
    set_smem(kern, sm);
    prof_begin(s);
    kern<<<1, TH, sm, s>>>(g, f, 0, 0, chat, 0, scale);
    prof_end(s, K_SPECTRUM, 8.0 * g.N + 16.0 * (double)((1 << g.lg_n) + 1), 0.0);
    return;
  }
  cplx<df64>* Y = reinterpret_cast<cplx<df64>*>(scratch);
  fs_forward<df64, GATHER_CIRC, double>(g, f, 0, 0, Y, 1, s, K_SPECTRUM, 8.0 * g.N);
  RowArgs ra{};
  ra.spec_out = chat;
  ra.natural = natural;
  ra.scale = scale;
  fs_row<df64, ROW_FWD_STORE>(g, Y, ra, 1, s, K_SPECTRUM, 16.0 * (double)((1 << g.lg_n) + 1));
}

void launch_spectrum64(const Geom& g, const double* f, cplx<double>* chat, int natural, float scale, void* scratch,
                       cudaStream_t s) {
  if (native_small(g)) {
    const size_t sm = (size_t)(1 << g.lg_n) * sizeof(cplx<double>);
    auto kern = k_rfft_small<double, TH, Lim<double>::MAXE, GATHER_CIRC, double>;
    set_smem(kern, sm);
    prof_begin(s);
    kern<<<1, TH, sm, s>>>(g, f, 0, 0, chat, 0, scale);
    prof_end(s, K_SPECTRUM, 8.0 * g.N + 16.0 * (double)((1 << g.lg_n) + 1), 0.0);
    return;
  }
  cplx<double>* Y = reinterpret_cast<cplx<double>*>(scratch);
  fs_forward<double, GATHER_CIRC, double>(g, f, 0, 0, Y, 1, s, K_SPECTRUM, 8.0 * g.N);
  RowArgs ra{};
  ra.spec_out = chat;
  ra.natural = natural;
  ra.scale = scale;
  fs_row<double, ROW_FWD_STORE>(g, Y, ra, 1, s, K_SPECTRUM, 16.0 * (double)((1 << g.lg_n) + 1));
}

template <class T, class Out>
static void hankel_impl(const Geom& g, const df64* U, int64_t ldu, const df64* V, int64_t ldv, const double* sigma,
                        const int* grp_off_dev, const int* grp_idx_dev, const int* grp_off_host,
                        const int* grp_idx_host, int m, Out* out, int64_t ldo, void* scratch, int rows,
                        int* dev_idx, bool small, double oscale, cudaStream_t s) {
  if (small) {
    constexpr int MAXE = Lim<T>::MAXE;
    const size_t sm = (size_t)(2 << g.lg_n) * sizeof(cplx<T>);
    auto kern = k_hankel_small<T, TH, MAXE, Out>;
    set_smem(kern, sm);
    prof_begin(s);
    kern<<<m, TH, sm, s>>>(g, U, ldu, V, ldv, sigma, grp_off_dev, grp_idx_dev, out, ldo, oscale);
    prof_end(s, K_HANKEL_SMALL, 8.0 * (double)(g.L + g.K) * grp_off_host[m] + 8.0 * (double)g.N * m, 0.0);
    return;
  }
  // Large M.  Groups in chunks of `rows`; within a chunk the components go in
  // rounds, round r holding the r-th member of every group that has one, so no
  // two batch rows of a launch add into the same accumulator.  Per round: the
  // forward FFTs of all its u' (spectra stored) and of all its v' (multiplied by
  // sigma and the stored u spectrum into the groups' accumulators), one launch
  // each; per chunk: one inverse of all its groups.
  const int64_t n = (int64_t)1 << g.lg_n;
  const int R = rows < 1 ? 1 : rows;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char* base = static_cast<char*>(scratch);
  cplx<T>* Y = reinterpret_cast<cplx<T>*>(base);
  cplx<df64>* su = reinterpret_cast<cplx<df64>*>(base + al((size_t)R * n * sizeof(cplx<T>)));
  cplx<df64>* acc = reinterpret_cast<cplx<df64>*>(reinterpret_cast<char*>(su) + al((size_t)R * (n + 1) * 16));
  // host list of (component, accumulator row) per round, uploaded once
  std::vector<int> idx;
  struct Round { int g0, gc, off, b; };
  std::vector<Round> plan;
  for (int g0 = 0; g0 < m; g0 += R) {
    const int gc = std::min(R, m - g0);
    int maxsz = 0;
    for (int gg = g0; gg < g0 + gc; ++gg) maxsz = std::max(maxsz, grp_off_host[gg + 1] - grp_off_host[gg]);
    if (maxsz == 0) {  // only empty groups: their reconstructions are zero
      for (int gg = g0; gg < g0 + gc; ++gg) cudaMemsetAsync(out + (int64_t)gg * ldo, 0, (size_t)g.N * sizeof(Out), s);
      continue;
    }
    plan.push_back({g0, gc, -1, 0});  // chunk marker (b = 0): clear, then rounds, then the inverse
    for (int r = 0; r < maxsz; ++r) {
      Round rd{g0, gc, (int)idx.size(), 0};
      std::vector<int> comps, accs;
      for (int gg = g0; gg < g0 + gc; ++gg)
        if (grp_off_host[gg + 1] - grp_off_host[gg] > r) {
          comps.push_back(grp_idx_host[grp_off_host[gg] + r]);
          accs.push_back(gg - g0);
        }
      rd.b = (int)comps.size();
      idx.insert(idx.end(), comps.begin(), comps.end());
      idx.insert(idx.end(), accs.begin(), accs.end());
      plan.push_back(rd);
    }
  }
  if (!idx.empty()) cudaMemcpyAsync(dev_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  for (size_t i = 0; i < plan.size(); ++i) {
    const Round& rd = plan[i];
    if (rd.b == 0) {
      cudaMemsetAsync(acc, 0, (size_t)rd.gc * (n + 1) * sizeof(cplx<df64>), s);
      continue;
    }
    const int* dcomp = dev_idx + rd.off;
    const int* dacc = dcomp + rd.b;
    fs_forward<T, GATHER_PAD, df64>(g, U, ldu, g.L, Y, rd.b, s, K_HANKEL_FS, 8.0 * g.L * rd.b, -1, dcomp);
    RowArgs ra{};
    ra.spec_out = su;
    ra.ld_spec = n + 1;
    ra.natural = 0;
    ra.scale = 1.0f;
    fs_row<T, ROW_FWD_STORE>(g, Y, ra, rd.b, s, K_HANKEL_FS, 0.0);
    fs_forward<T, GATHER_PAD, df64>(g, V, ldv, g.K, Y, rd.b, s, K_HANKEL_FS, 8.0 * g.K * rd.b, -1, dcomp);
    RowArgs rb{};
    rb.spec_in = su;
    rb.spec_out = acc;
    rb.ld_spec = n + 1;
    rb.weight = sigma;
    rb.weight_of_row = dcomp;
    rb.out_of_row = dacc;
    fs_row<T, ROW_FWD_MUL_ACC>(g, Y, rb, rd.b, s, K_HANKEL_FS, 0.0);
    const bool last_round = i + 1 == plan.size() || plan[i + 1].b == 0;
    if (last_round) {
      RowArgs rc{};
      rc.spec_in = acc;
      rc.ld_spec = n + 1;
      fs_row<T, ROW_INV_LOAD>(g, Y, rc, rd.gc, s, K_HANKEL_FS, 0.0);
      fs_inverse<T, OUT_HANKEL, Out>(g, Y, out + (int64_t)rd.g0 * ldo, ldo, 0, 0, 1.0f / (2.0f * (float)n), rd.gc, s,
                                     K_HANKEL_FS, 8.0 * (double)g.N * rd.gc, -1, oscale);
    }
  }
}

size_t hankel_scratch_bytes(const Geom& g, int prec, int rows) {
  const int64_t n = (int64_t)1 << g.lg_n;
  const bool f32 = prec == PREC_F32C;
  if (((int64_t)2 << g.lg_n) <= (f32 ? Lim<float>::MAXE : Lim<df64>::MAXE)) return 0;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t R = rows < 1 ? 1 : rows;
  return al(R * n * (f32 ? sizeof(cplx<float>) : sizeof(cplx<df64>))) + al(R * (n + 1) * 16) + R * (n + 1) * 16;
}

void launch_hankel(const Geom& g, int prec, const df64* U, int64_t ldu, const df64* V, int64_t ldv,
                   const double* sigma, const int* grp_off_dev, const int* grp_idx_dev, const int* grp_off_host,
                   const int* grp_idx_host, int m, double* out, int64_t ldo, void* scratch, int rows, int* dev_idx,
                   double oscale, cudaStream_t s) {
  // the small kernel holds two length-n buffers
  if (prec == PREC_F32C) {
    const bool sm = ((int64_t)2 << g.lg_n) <= Lim<float>::MAXE;
    hankel_impl<float, double>(g, U, ldu, V, ldv, sigma, grp_off_dev, grp_idx_dev, grp_off_host, grp_idx_host, m,
                               out, ldo, scratch, rows, dev_idx, sm, oscale, s);
  } else {
    const bool sm = ((int64_t)2 << g.lg_n) <= Lim<df64>::MAXE;
    hankel_impl<df64, double>(g, U, ldu, V, ldv, sigma, grp_off_dev, grp_idx_dev, grp_off_host, grp_idx_host, m, out,
                              ldo, scratch, rows, dev_idx, sm, oscale, s);
  }
}

// ---- autotuner of the four-step tiles
template <class F> static float time_min(F run, cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  run();  // warm-up (and the shared-memory opt-in)
  float ms = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    for (int i = 0; i < 4; ++i) run();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms = std::min(ms, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

// fastest column tile (lg_cb | thread index << 8) of a pass
template <class T>
static int tune_one(const Geom& g, int pass, const df64* x, df64* y, cplx<T>* Y, cudaStream_t s) {
  const int maxcb = col_lg_cb(g, Lim<T>::COLE);
  int best = maxcb | (1 << 8);
  float best_ms = 1e30f;
  for (int th = 0; th < 3; ++th) {
    for (int cb = 0; cb <= maxcb; ++cb) {
      const int tile = cb | (th << 8);
      const float ms = time_min(
          [&]() {
            if (pass == 0) fs_forward<T, GATHER_X, df64>(g, x, 0, 0, Y, 1, s, K_MISC, 0.0, tile);
            else fs_inverse<T, OUT_SLICE, df64>(g, Y, y, 0, 0, g.L, 1.0f, 1, s, K_MISC, 0.0, tile);
          },
          s);
      if (ms < best_ms) {
        best_ms = ms;
        best = tile;
      }
    }
  }
  return best;
}

// fastest threads per CTA of the product's row pass: 0 (256) or 1 (512)
template <class T> static int tune_row(const Geom& g, cplx<T>* Y, const cplx<df64>* chat, cudaStream_t s) {
  if (!row_mv_applies<T>(g, Y, chat)) return 0;
  RowArgs ra{};
  ra.chat = chat;
  const float a = time_min([&]() { fs_row<T, ROW_MATVEC>(g, Y, ra, 1, s, K_MISC, 0.0, 256); }, s);
  const float b = time_min([&]() { fs_row<T, ROW_MATVEC>(g, Y, ra, 1, s, K_MISC, 0.0, 512); }, s);
  return b < a ? 1 : 0;
}

int autotune_fourstep(const Geom& g, int prec, cudaStream_t s) {
  tune_table_init();
  if (small_path(g, prec)) return 0;
  const int slot = prec == PREC_F32C ? 0 : 1;
  if (g_tuned_cb[slot][0][g.lg_n].load() >= 0 && g_tuned_cb[slot][1][g.lg_n].load() >= 0 &&
      g_tuned_row[slot][g.lg_n].load() >= 0)
    return 0;
  const int64_t n = (int64_t)1 << g.lg_n;
  void* buf = nullptr;
  // every carved piece starts on a 256-byte boundary (the row pass stages Y and the spectrum with
  // bulk copies, which need 16-byte aligned addresses)
  const size_t xb = ((size_t)(g.K + g.L + 8) * sizeof(df64) + 255) / 256 * 256;
  const size_t yb = ((size_t)n * sizeof(cplx<df64>) + 255) / 256 * 256, cb = (size_t)(n + 1) * sizeof(cplx<df64>);
  cudaError_t e = cudaMallocAsync(&buf, xb + yb + cb, s);
  if (e != cudaSuccess) return (int)e;
  cudaMemsetAsync(buf, 0, xb + yb + cb, s);
  df64* x = static_cast<df64*>(buf);
  df64* y = x + g.K + 4;
  void* Yv = static_cast<char*>(buf) + xb;
  const cplx<df64>* chat = reinterpret_cast<const cplx<df64>*>(static_cast<char*>(buf) + xb + yb);
  prof_suppress(true);
  int f, i, r;
  if (slot == 0) {
    f = tune_one<float>(g, 0, x, y, static_cast<cplx<float>*>(Yv), s);
    i = tune_one<float>(g, 1, x, y, static_cast<cplx<float>*>(Yv), s);
    r = tune_row<float>(g, static_cast<cplx<float>*>(Yv), chat, s);
  } else {
    f = tune_one<df64>(g, 0, x, y, static_cast<cplx<df64>*>(Yv), s);
    i = tune_one<df64>(g, 1, x, y, static_cast<cplx<df64>*>(Yv), s);
    r = tune_row<df64>(g, static_cast<cplx<df64>*>(Yv), chat, s);
  }
  prof_suppress(false);
  g_tuned_cb[slot][0][g.lg_n].store(f);
  g_tuned_cb[slot][1][g.lg_n].store(i);
  g_tuned_row[slot][g.lg_n].store(r);
  cudaFreeAsync(buf, s);
  return (int)cudaGetLastError();
}

int tuned_tiling(int prec, int lg_n, int pass) {
  tune_table_init();
  if (lg_n < 0 || lg_n >= 32 || pass < 0 || pass > 1) return -1;
  const int v = g_tuned_cb[prec == PREC_F32C ? 0 : 1][pass][lg_n].load();
  return v < 0 ? v : (v & 0xff);
}

int tuned_threads(int prec, int lg_n, int pass) {
  tune_table_init();
  if (lg_n < 0 || lg_n >= 32 || pass < 0 || pass > 2) return 0;
  const int slot = prec == PREC_F32C ? 0 : 1;
  if (pass == 2) {
    const int r = g_tuned_row[slot][lg_n].load();
    return r < 0 ? 0 : (r == 1 ? 512 : 256);
  }
  const int v = g_tuned_cb[slot][pass][lg_n].load();
  return v < 0 ? 0 : COL_THREADS[(v >> 8) & 3];
}

size_t spectral_scratch_bytes(const Geom& g) {
  const int64_t n = (int64_t)1 << g.lg_n;
  // Y (n complex df64) + u spectrum and accumulator (n+1 complex df64 each)
  return (size_t)(n + 2 * (n + 1)) * sizeof(cplx<df64>);
}

}  // namespace ssa
