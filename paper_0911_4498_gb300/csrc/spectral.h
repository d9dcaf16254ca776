// Host-side interface of the spectral kernels (spectral.cu).
#pragma once
#include <type_traits>
#include "common.cuh"

namespace ssa {

enum { PREC_F64 = 0, PREC_F32C = 1, PREC_NATIVE64 = 2 };

// Largest n = M / 2 of a product run by one CTA in shared memory (128 KB of
// complex values), per arithmetic type; larger n takes the four-step kernels.
constexpr int SMALL_MAXE_F32 = 16384;
constexpr int SMALL_MAXE_DF64 = 8192;
enum { GATHER_X = 0, GATHER_XT = 1, GATHER_CIRC = 2, GATHER_PAD = 3 };
enum { ROW_MATVEC = 0, ROW_FWD_STORE = 1, ROW_FWD_MUL_ACC = 2, ROW_INV_LOAD = 3 };
enum { OUT_SLICE = 0, OUT_HANKEL = 1 };

// FFT geometry of one (N, L) plan.  M = 2^(lg_n+1) >= N.  Small plans (one
// CTA per transform) use tw = W_n^m; four-step plans split n = n1 * n2 with
// n1 = 2^lg_n1 <= n2 = 2^lg_n2 and use tw = W_{n2}^m.  tA/tB give
// W_M^m = tA[m >> tws] * tB[m & (2^tws - 1)].
struct Geom {
  int64_t N, L, K, M;
  int lg_n, lg_n1, lg_n2;
  const cplx<df64>* tw;
  int lg_P;
  const cplx<df64>* tA;
  const cplx<df64>* tB;
  int tws;
  int twshift;  // the two-level table is for M << twshift (batched series share the largest table)
  // IEEE-double copies of the tables for the native-FP64 products (may be null)
  const cplx<double>* tw64;
  const cplx<double>* tA64;
  const cplx<double>* tB64;
};

// table pointers of the arithmetic type T
template <class T> SSA_HD const tab_t<T>* g_tw(const Geom& g) {
  if constexpr (std::is_same<T, double>::value) return g.tw64; else return g.tw;
}
template <class T> SSA_HD const tab_t<T>* g_tA(const Geom& g) {
  if constexpr (std::is_same<T, double>::value) return g.tA64; else return g.tA;
}
template <class T> SSA_HD const tab_t<T>* g_tB(const Geom& g) {
  if constexpr (std::is_same<T, double>::value) return g.tB64; else return g.tB;
}

// Spectrum pointers are of the table type tab_t<T> of the kernel's arithmetic
// type T (double-float for FP32 and df64 arithmetic, double for native FP64).
struct RowArgs {
  const void* chat;            // ROW_MATVEC: scaled spectrum, four-step order
  const void* spec_in;         // ROW_FWD_MUL_ACC / ROW_INV_LOAD input spectrum
  void* spec_out;              // ROW_FWD_STORE / ROW_FWD_MUL_ACC output spectrum
  int64_t ld_spec;             // batch stride of spec_in / spec_out
  int natural;                 // ROW_FWD_STORE: natural index order (else four-step)
  float scale;                 // ROW_FWD_STORE: multiply W by this power of two
  const double* weight;        // ROW_FWD_MUL_ACC: sigma array on the device
  int weight_idx;
  // ROW_FWD_MUL_ACC over a batch: per batch row y, the weight index (component)
  // and the spec_out row (group accumulator); null: weight_idx and row y
  const int* weight_of_row;
  const int* out_of_row;
};

bool small_path(const Geom& g, int prec);
// copy the fault word of the spectral kernels (nonzero once a bounded wait
// for a TMA bulk copy ran out) to *host, ordered on s
int spectral_fault_read(unsigned* host, cudaStream_t s);
// Time the column tilings of the four-step passes for this n and precision
// once per process (synchronises s); returns a cudaError_t value.
int autotune_fourstep(const Geom& g, int prec, cudaStream_t s);
// tuned log2(columns per CTA) for (precision, lg_n, pass 0 = forward / 1 = inverse), -1 if not tuned
int tuned_tiling(int prec, int lg_n, int pass);
// tuned threads per CTA for (precision, lg_n, pass 0 = forward columns / 1 = inverse
// columns / 2 = the product's rows), 0 if not tuned
int tuned_threads(int prec, int lg_n, int pass);
size_t spectral_scratch_bytes(const Geom& g);
void launch_matvec_df(const Geom& g, int prec, int transpose, const df64* x, int64_t ldx, df64* y, int64_t ldy,
                      int batch, const cplx<df64>* chat, void* scratch, cudaStream_t s);
void launch_matvec_d(const Geom& g, int prec, int transpose, const double* x, int64_t ldx, double* y, int64_t ldy,
                     int batch, const cplx<df64>* chat, void* scratch, cudaStream_t s);
void launch_spectrum(const Geom& g, const double* f, cplx<df64>* chat, int natural, float scale, void* scratch,
                     cudaStream_t s);
// native-FP64 spectrum (double tables), natural order or four-step order as above
void launch_spectrum64(const Geom& g, const double* f, cplx<double>* chat, int natural, float scale, void* scratch,
                       cudaStream_t s);
// the native-FP64 product runs in one CTA (else four-step, n complex doubles of scratch per vector)
bool native_small(const Geom& g);
// y_j = X x_j in native FP64 with the double spectrum (Rayleigh-quotient refinement)
void launch_matvec_native(const Geom& g, int transpose, const double* x, int64_t ldx, double* y, int64_t ldy,
                          int batch, const cplx<double>* chat, void* scratch, cudaStream_t s);
// Grouped Hankelization; every output value is multiplied by oscale (a power
// of two: sigma may be passed scaled into range and the result scaled back).
// Four-step sizes transform the components of up to `rows` groups per launch
// (scratch of hankel_scratch_bytes(g, prec, rows) bytes, 256-byte aligned, and
// dev_idx, device room for 2 * (number of grouped components) ints); one CTA
// per group at the single-CTA sizes (scratch and dev_idx unused).
void launch_hankel(const Geom& g, int prec, const df64* U, int64_t ldu, const df64* V, int64_t ldv,
                   const double* sigma, const int* grp_off_dev, const int* grp_idx_dev, const int* grp_off_host,
                   const int* grp_idx_host, int m, double* out, int64_t ldo, void* scratch, int rows, int* dev_idx,
                   double oscale, cudaStream_t s);
// bytes of Hankelization scratch for `rows` groups per launch (0 at the single-CTA sizes)
size_t hankel_scratch_bytes(const Geom& g, int prec, int rows);

}  // namespace ssa
