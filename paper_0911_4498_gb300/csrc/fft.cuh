// In-shared-memory batched complex FFT for one CTA, and the real-FFT
// packing used by Algorithms 2-4.
//
// cta_fft: `count` transforms of power-of-two length `len`, stored back to
// back in shared memory.  Stockham autosort with radix-4 stages and one
// radix-2 stage when log2(len) is odd, in the formulation of Govindaraju et
// al. (SC'08): butterfly j of a stage with span Ns reads x[j + r*len/R],
// twiddles it by W_{Ns R}^{r (j mod Ns)}, does an R-point DFT and writes
// y[(j/Ns) Ns R + (j mod Ns) + r Ns].  Each thread keeps its butterflies in
// registers across a barrier, so the transform runs in place in one buffer.
// Output is in natural order; the inverse is unnormalised.
//
// Real FFT of length M = 2n by a half-length complex FFT: pack
// z_t = w_{2t} + i w_{2t+1}, Z = FFT_n(z), then for k in [0, n]
//   W_k = 1/2 (Z_k + conj Z_{n-k}) - i/2 W_M^k (Z_k - conj Z_{n-k}).
// Inverse: Z'_k = 1/2 (P_k + conj P_{n-k}) + i/2 W_M^{-k} (P_k - conj P_{n-k}),
// z' = IFFT_n(Z'), p_{2t} = Re z'_t, p_{2t+1} = Im z'_t.  The helpers below
// return twice these values; constant factors are folded into the stored
// spectrum of the series.
#pragma once
#include <type_traits>
#include "common.cuh"

namespace ssa {

template <class T, bool INV>
SSA_D void bfly2(cplx<T>& a, cplx<T>& b) {
  cplx<T> s = c_add(a, b);
  b = c_sub(a, b);
  a = s;
}

template <class T, bool INV>
SSA_D void bfly4(cplx<T>& x0, cplx<T>& x1, cplx<T>& x2, cplx<T>& x3) {
  cplx<T> a = c_add(x0, x2), b = c_sub(x0, x2);
  cplx<T> c = c_add(x1, x3), d = c_sub(x1, x3);
  // forward: W_4 = -i ; inverse: +i
  cplx<T> dd = INV ? c_mul_i(d) : c_mul_mi(d);
  x0 = c_add(a, c);
  x2 = c_sub(a, c);
  x1 = c_add(b, dd);
  x3 = c_sub(b, dd);
}

// Twiddle accessors: W_P^m from the table in global memory (read-only path),
// or from a copy of it in shared memory.
template <class T> struct TwGlobal {
  const tab_t<T>* p;
  SSA_D cplx<T> operator()(int64_t m) const { return tw_load<T>(p, m); }
};
template <class T> struct TwShared {
  const tab_t<T>* p;
  SSA_D cplx<T> operator()(int64_t m) const {
    const tab_t<T> v = p[m];
    if constexpr (std::is_same<T, float>::value) return mk(v.re.hi + v.re.lo, v.im.hi + v.im.lo);
    else return v;
  }
};

// One Stockham stage of radix R.  ilog2 arguments avoid integer division.
// Transform t starts at buf + t * tstride (tstride >= len; padding between
// transforms spreads a column-major tile over the shared-memory banks).
template <class T, int R, int THREADS, int MAXE, bool INV, class TW = TwGlobal<T>>
SSA_D void fft_stage(cplx<T>* buf, int lg_len, int count, int lg_ns, TW tw, int lg_P, int tstride) {
  constexpr int MAXB = (MAXE / R + THREADS - 1) / THREADS;
  const int lg_nbp = lg_len - (R == 4 ? 2 : 1);  // log2 butterflies per transform
  const int nb = count << lg_nbp;
  const int len = 1 << lg_len;
  const int nbp = 1 << lg_nbp;
  const int ns = 1 << lg_ns;
  const int tw_shift = lg_P - lg_ns - (R == 4 ? 2 : 1);  // P / (Ns R) as a shift
  cplx<T> v[MAXB][R];
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int jj = threadIdx.x + q * THREADS;
    if (jj < nb) {
      const int t = jj >> lg_nbp;
      const int j = jj & (nbp - 1);
      const cplx<T>* base = buf + (size_t)t * tstride;
      const int jm = j & (ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cplx<T> x = base[j + r * nbp];
        if (r > 0 && jm != 0) {
          cplx<T> w = tw((int64_t)(r * jm) << tw_shift);
          x = INV ? c_mul_conj(x, w) : c_mul(x, w);
        }
        v[q][r] = x;
      }
      if (R == 4) bfly4<T, INV>(v[q][0], v[q][1], v[q][2], v[q][3]);
      else bfly2<T, INV>(v[q][0], v[q][1]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int jj = threadIdx.x + q * THREADS;
    if (jj < nb) {
      const int t = jj >> lg_nbp;
      const int j = jj & (nbp - 1);
      cplx<T>* base = buf + (size_t)t * tstride;
      const int jm = j & (ns - 1);
      const int idx = ((j >> lg_ns) << (lg_ns + (R == 4 ? 2 : 1))) + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) base[idx + r * ns] = v[q][r];
    }
  }
  __syncthreads();
  (void)len;
}

// Batched in-place FFT; caller must __syncthreads() before (data loaded) —
// the routine ends with a barrier.
template <class T, int THREADS, int MAXE, bool INV, class TW>
SSA_D void cta_fft_tw(cplx<T>* buf, int lg_len, int count, TW tw, int lg_P, int tstride = 0) {
  if (tstride <= 0) tstride = 1 << lg_len;
  int lg_ns = 0;
  while (lg_len - lg_ns >= 2) {
    fft_stage<T, 4, THREADS, MAXE, INV, TW>(buf, lg_len, count, lg_ns, tw, lg_P, tstride);
    lg_ns += 2;
  }
  if (lg_len - lg_ns == 1) fft_stage<T, 2, THREADS, MAXE, INV, TW>(buf, lg_len, count, lg_ns, tw, lg_P, tstride);
}
template <class T, int THREADS, int MAXE, bool INV>
SSA_D void cta_fft(cplx<T>* buf, int lg_len, int count, const tab_t<T>* tw, int lg_P) {
  cta_fft_tw<T, THREADS, MAXE, INV>(buf, lg_len, count, TwGlobal<T>{tw}, lg_P);
}

// Real-FFT post-processing for the pair (k, n-k); returns 2 W_k and 2 W_{n-k}
// (for k = 0 the second output is 2 W_n).  twk = W_M^k.
template <class T>
SSA_D void rfft_post(cplx<T> zk, cplx<T> znk, cplx<T> twk, cplx<T>& wk, cplx<T>& wnk) {
  cplx<T> bc = c_conj(znk);
  cplx<T> e = c_add(zk, bc);
  cplx<T> o = c_mul_mi(c_sub(zk, bc));
  cplx<T> t = c_mul(twk, o);
  wk = c_add(e, t);
  wnk = c_conj(c_sub(e, t));
}

// Inverse pre-processing for the pair (k, n-k); returns 2 Z'_k and 2 Z'_{n-k}
// (for k = 0, pk = P_0 and pnk = P_n; only zk is meaningful).
template <class T>
SSA_D void irfft_pre(cplx<T> pk, cplx<T> pnk, cplx<T> twk, cplx<T>& zk, cplx<T>& znk) {
  cplx<T> pc = c_conj(pnk);
  cplx<T> s = c_add(pk, pc);
  cplx<T> d = c_sub(pk, pc);
  cplx<T> t = c_mul_i(c_mul_conj(d, twk));
  zk = c_add(s, t);
  znk = c_conj(c_sub(s, t));
}

// W_M^m from a two-level table: tA[m >> s] * tB[m & (2^s - 1)].
template <class T>
SSA_D cplx<T> twiddle_M(const tab_t<T>* tA, const tab_t<T>* tB, int s, int64_t m) {
  cplx<T> a = tw_load<T>(tA, m >> s);
  cplx<T> b = tw_load<T>(tB, m & ((1 << s) - 1));
  return c_mul(a, b);
}

// Spectrum multiply: FP32 data times a double-float spectrum keeps the
// spectrum's extra bits (compensated product); df64 data multiply in df64.
SSA_D cplx<float> mul_spec(cplx<float> w, cplx<df64> c) {
  float re = fmaf(w.re, c.re.hi, fmaf(-w.im, c.im.hi, fmaf(w.re, c.re.lo, -w.im * c.im.lo)));
  float im = fmaf(w.re, c.im.hi, fmaf(w.im, c.re.hi, fmaf(w.re, c.im.lo, w.im * c.re.lo)));
  return mk(re, im);
}
SSA_D cplx<df64> mul_spec(cplx<df64> w, cplx<df64> c) { return c_mul(w, c); }
SSA_D cplx<double> mul_spec(cplx<double> w, cplx<double> c) { return c_mul(w, c); }

}  // namespace ssa
