// Shared device-side definitions for the fast-SSA CUDA library (sm_103a).
//
// Arithmetic types.  GB300's FP64 pipe issues roughly 1/68 of the FP32 rate
// (DFMA ~1.0 TFLOP/s, DADD and F2F.F64 ~0.5-0.6 Tops/s measured), so every
// step that needs double-precision accuracy computes in "double-float"
// (df64): an unevaluated sum hi + lo of two floats, ~48 significant bits.
// The error-free building blocks are Knuth's TwoSum, Dekker's Fast2Sum and
// the FMA-based TwoProduct (Dekker 1971; Ogita, Rump, Oishi 2005); division
// is Dekker's long division with one correction, square root is one Newton
// step on the FP32 root (Karp & Markstein 1997).
//
// Storage: a df64 value is a float2 {hi, lo} (8 bytes, same as a double),
// so df64 vectors stream with the same HBM traffic as FP64 ones.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SSA_HD __host__ __device__ __forceinline__
#define SSA_D __device__ __forceinline__

struct __align__(8) df64 {
  float hi, lo;
};

SSA_HD df64 make_df(float h, float l) { df64 r; r.hi = h; r.lo = l; return r; }
SSA_HD df64 df_zero() { return make_df(0.f, 0.f); }

// exact: s + e == a + b
SSA_HD df64 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return make_df(s, e);
}
// exact when |a| >= |b| (or a == 0)
SSA_HD df64 fast_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return make_df(s, e);
}
// exact: p + e == a * b
SSA_HD df64 two_prod(float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  return make_df(p, e);
}

SSA_HD df64 df_add(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  float e = s.lo + (a.lo + b.lo);
  return fast_two_sum(s.hi, e);
}
SSA_HD df64 df_neg(df64 a) { return make_df(-a.hi, -a.lo); }
SSA_HD df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }
SSA_HD df64 df_mul(df64 a, df64 b) {
  df64 p = two_prod(a.hi, b.hi);
  float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}
SSA_HD df64 df_mul_f(df64 a, float b) {
  df64 p = two_prod(a.hi, b);
  float e = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, e);
}
// a*b + c with one normalisation
SSA_HD df64 df_fma(df64 a, df64 b, df64 c) {
  df64 p = two_prod(a.hi, b.hi);
  df64 s = two_sum(p.hi, c.hi);
  float e = s.lo + (p.lo + c.lo) + fmaf(a.hi, b.lo, a.lo * b.hi);
  return fast_two_sum(s.hi, e);
}
// exact scaling by a power of two
SSA_HD df64 df_scale(df64 a, float p2) { return make_df(a.hi * p2, a.lo * p2); }
SSA_HD df64 df_div(df64 a, df64 b) {
  float q1 = a.hi / b.hi;
  df64 p = two_prod(q1, b.hi);
  float r = ((a.hi - p.hi) - p.lo) + a.lo - q1 * b.lo;
  float q2 = r / b.hi;
  return fast_two_sum(q1, q2);
}
SSA_HD df64 df_sqrt(df64 a) {
  if (!(a.hi > 0.f)) return df_zero();
  float s = sqrtf(a.hi);
  df64 ss = two_prod(s, s);
  float r = ((a.hi - ss.hi) - ss.lo) + a.lo;
  return fast_two_sum(s, r / (2.f * s));
}
SSA_HD df64 df_abs(df64 a) { return a.hi < 0.f ? df_neg(a) : a; }
SSA_HD bool df_lt(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
SSA_HD bool df_gt(df64 a, df64 b) { return df_lt(b, a); }

// conversions at the API boundary (not on hot loops: F2F.F64 is slow on GB300)
SSA_HD df64 df_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return make_df(h, l);
}
SSA_HD double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------------------
// Generic scalar interface so FFT code can be written once for float and df64.
SSA_HD float s_add(float a, float b) { return a + b; }
SSA_HD float s_sub(float a, float b) { return a - b; }
SSA_HD float s_mul(float a, float b) { return a * b; }
SSA_HD float s_neg(float a) { return -a; }
SSA_HD float s_scale(float a, float p2) { return a * p2; }
SSA_HD double s_add(double a, double b) { return a + b; }
SSA_HD double s_sub(double a, double b) { return a - b; }
SSA_HD double s_mul(double a, double b) { return a * b; }
SSA_HD double s_neg(double a) { return -a; }
SSA_HD double s_scale(double a, float p2) { return a * (double)p2; }
SSA_HD df64 s_add(df64 a, df64 b) { return df_add(a, b); }
SSA_HD df64 s_sub(df64 a, df64 b) { return df_sub(a, b); }
SSA_HD df64 s_mul(df64 a, df64 b) { return df_mul(a, b); }
SSA_HD df64 s_neg(df64 a) { return df_neg(a); }
SSA_HD df64 s_scale(df64 a, float p2) { return df_scale(a, p2); }

template <class T> struct scal;
template <> struct scal<float> {
  SSA_HD static float zero() { return 0.f; }
  SSA_HD static float from_df(df64 a) { return a.hi + a.lo; }
  SSA_HD static float from_double(double x) { return (float)x; }
  SSA_HD static df64 to_df(float a) { return make_df(a, 0.f); }
};
template <> struct scal<df64> {
  SSA_HD static df64 zero() { return df_zero(); }
  SSA_HD static df64 from_df(df64 a) { return a; }
  SSA_HD static df64 from_double(double x) { return df_from_double(x); }
  SSA_HD static df64 to_df(df64 a) { return a; }
};

template <> struct scal<double> {
  SSA_HD static double zero() { return 0.0; }
  SSA_HD static double from_df(df64 a) { return (double)a.hi + (double)a.lo; }
  SSA_HD static double from_double(double x) { return x; }
  SSA_HD static df64 to_df(double a) { return df_from_double(a); }
};

template <class T> struct cplx {
  T re, im;
};
static_assert(sizeof(cplx<df64>) == 16, "cplx<df64> must be 16 bytes");
template <class T> SSA_HD cplx<T> mk(T r, T i) { cplx<T> z; z.re = r; z.im = i; return z; }
template <class T> SSA_HD cplx<T> c_add(cplx<T> a, cplx<T> b) { return mk(s_add(a.re, b.re), s_add(a.im, b.im)); }
template <class T> SSA_HD cplx<T> c_sub(cplx<T> a, cplx<T> b) { return mk(s_sub(a.re, b.re), s_sub(a.im, b.im)); }
template <class T> SSA_HD cplx<T> c_conj(cplx<T> a) { return mk(a.re, s_neg(a.im)); }
// multiply by +i (or -i)
template <class T> SSA_HD cplx<T> c_mul_i(cplx<T> a) { return mk(s_neg(a.im), a.re); }
template <class T> SSA_HD cplx<T> c_mul_mi(cplx<T> a) { return mk(a.im, s_neg(a.re)); }
template <class T> SSA_HD cplx<T> c_scale(cplx<T> a, float p2) { return mk(s_scale(a.re, p2), s_scale(a.im, p2)); }
SSA_HD cplx<float> c_mul(cplx<float> a, cplx<float> b) {
  return mk(fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re));
}
SSA_HD cplx<double> c_mul(cplx<double> a, cplx<double> b) {
  return mk(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
SSA_HD cplx<df64> c_mul(cplx<df64> a, cplx<df64> b) {
  return mk(df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re)));
}
// a * conj(b)
template <class T> SSA_HD cplx<T> c_mul_conj(cplx<T> a, cplx<T> b) { return c_mul(a, c_conj(b)); }

// Twiddle tables and spectra are stored in df64 (float2 pairs for re and im)
// for the FP32 and df64 paths -- FP32 code reads the rounded value -- and in
// IEEE double for the native-FP64 path.
template <class T> struct tabt { using type = cplx<df64>; };
template <> struct tabt<double> { using type = cplx<double>; };
template <class T> using tab_t = typename tabt<T>::type;

template <class T> SSA_D cplx<T> tw_load(const tab_t<T>* tab, int64_t m);
template <> SSA_D cplx<df64> tw_load<df64>(const cplx<df64>* tab, int64_t m) {
  float4 v = __ldg(reinterpret_cast<const float4*>(tab) + m);
  return mk(make_df(v.x, v.y), make_df(v.z, v.w));
}
template <> SSA_D cplx<double> tw_load<double>(const cplx<double>* tab, int64_t m) {
  double2 v = __ldg(reinterpret_cast<const double2*>(tab) + m);
  return mk(v.x, v.y);
}
template <> SSA_D cplx<float> tw_load<float>(const cplx<df64>* tab, int64_t m) {
  float4 v = __ldg(reinterpret_cast<const float4*>(tab) + m);
  return mk(v.x + v.y, v.z + v.w);
}

// Status word shared by device code and host: bit flags, never traps.
enum : uint32_t {
  SSA_DEV_OK = 0u,
  SSA_DEV_NONFINITE = 1u,
  SSA_DEV_JACOBI_NOCONV = 2u,
  SSA_DEV_BREAKDOWN = 4u,
};
