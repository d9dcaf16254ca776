// The fused lane-owned reorthogonalisation pass (section 3.2.2), in a file of
// its own so that its source can be identified independently of the
// launchers in cgs.cu.  Double-float (df64) throughout.
#pragma once
#include "lanczos.h"
#include "lanczos_dev.cuh"

namespace ssa {

// Fused CGS pass over Q (dim x ncols column-major, ncols <= 8 * CPW):
//   UPD:  w <- w - Q h          (h read from memory)
//   PROJ: part[block][c] = sum over the block's tiles of Q[tile, c] . w[tile]
//   always: part[block][ncols] = w.w over the block's tiles (after UPD)
// Persistent blocks walk tiles of 64 rows.  Warp wp owns the columns
// c = wp + 8m (m < CPW) and lane l the rows 2l, 2l+1 of every tile, so each
// lane stages (16-byte cp.async, NST tiles deep) and reads back only the
// pieces it copied itself: the basis tiles need no barrier.  (Requesting
// tiles further ahead into L2 with bulk prefetches measured slower in every
// pass.)  Under UPD every warp forms
// the partial row sums Q[rows, its columns] h[its columns]; after one barrier
// the first 64 threads add the eight partials of their row in warp order and
// write x = w - Q h (to shared memory when PROJ follows, and to w).  Under
// PROJ every lane accumulates its columns' products with its two rows of x
// over all the block's tiles in registers (lazy double-float accumulators);
// one warp reduction per column at the end.  Rows of w are prefetched into
// registers one tile ahead.  The projection after an update needs one more
// barrier (x visible); update-only passes double-buffer the partials instead.
constexpr int LR = 64;  // rows per tile: 32 lanes x 2 rows
template <bool UPD, bool PROJ, int CPW, int NST>
__global__ void __launch_bounds__(256, (CPW <= 13 ? 2 : 1))
    k_cgs_lanes(const df64* __restrict__ Q, int64_t ldq, int ncols, df64* __restrict__ w, int64_t dim,
                const df64* __restrict__ h, df64* __restrict__ part, int ldp, int ntiles, const int* flag) {
  if (flag && *flag == 0) return;
  constexpr int NRED = (UPD && !PROJ) ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) df64 red[NRED][8][LR];
  __shared__ __align__(16) df64 xs[LR];
  __shared__ df64 nred[8];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  df64* st0 = reinterpret_cast<df64*>(smem_raw);
  const int stage_elems = ncols * LR;
  // this warp's columns: c = wp + 8m for m < mycols (warp-uniform; the unrolled column
  // loops stop there instead of predicating the unused slots)
  const int mycols = ncols > wp ? (ncols - wp + 7) >> 3 : 0;
  df64 hr[CPW];
  dacc acc[CPW];
#pragma unroll
  for (int m = 0; m < CPW; ++m) {
    hr[m] = (UPD && m < mycols) ? h[wp + 8 * m] : df_zero();
    acc[m] = dacc_zero();
  }
  dacc nacc = dacc_zero();
  const df64* qlane = Q + (int64_t)wp * ldq + 2 * lane;
  const int64_t qstep = 8 * ldq;
  auto issue = [&](int stg, int tile) {  // this lane's 16-byte pieces of the tile (column c at c * LR)
    df64* st = st0 + stg * stage_elems + wp * LR + 2 * lane;
    const int64_t r0 = (int64_t)tile * LR;
    const bool ok = r0 + 2 * lane < dim;
#pragma unroll
    for (int m = 0; m < CPW; ++m) {
      if (m >= mycols) break;
      cp_async16(st + 8 * m * LR, ok ? (const void*)(qlane + m * qstep + r0) : (const void*)Q, ok);
    }
  };
  // rows of w: under UPD the first 64 threads hold one row each (plain loads: w is written
  // by this pass); otherwise every lane holds its two rows (read-only path)
  auto wrow = [&](int tile) -> df64 {
    const int64_t row = (int64_t)tile * LR + tid;
    return row < dim ? w[row] : df_zero();
  };
  auto wpair = [&](int tile) -> float4 { return ld_pair(w, (int64_t)tile * LR + 2 * lane, dim); };
  for (int p = 0; p < NST - 1; ++p) {
    const int t = blockIdx.x + p * gridDim.x;
    if (t < ntiles) issue(p, t);
    cp_async_commit();
  }
  df64 wr = df_zero();
  float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (blockIdx.x < ntiles) {
    if (UPD) {
      if (tid < LR) wr = wrow(blockIdx.x);
    } else {
      wv = wpair(blockIdx.x);
    }
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int ahead = tile + (NST - 1) * gridDim.x;
    if (ahead < ntiles) issue((it + NST - 1) % NST, ahead);
    cp_async_commit();
    const int nxt = tile + gridDim.x;
    df64 wr_n = wr;
    float4 wv_n = wv;
    if (nxt < ntiles) {
      if (UPD) {
        if (tid < LR) wr_n = wrow(nxt);
      } else {
        wv_n = wpair(nxt);
      }
    }
    cp_async_wait<NST - 1>();
    const df64* sl = st0 + (it % NST) * stage_elems + wp * LR + 2 * lane;
    const int64_t r0 = (int64_t)tile * LR;
    if (UPD) {
      dacc a0 = dacc_zero(), a1 = dacc_zero();
#pragma unroll
      for (int m = 0; m < CPW; ++m) {
        if (m >= mycols) break;
        const float4 v = *reinterpret_cast<const float4*>(sl + 8 * m * LR);
        dacc_fma(a0, make_df(v.x, v.y), hr[m]);
        dacc_fma(a1, make_df(v.z, v.w), hr[m]);
      }
      const df64 s0 = dacc_val(a0), s1 = dacc_val(a1);
      df64(*rb)[LR] = red[NRED == 2 ? (it & 1) : 0];
      *reinterpret_cast<float4*>(&rb[wp][2 * lane]) = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
      __syncthreads();
      if (tid < LR) {
        df64 s = rb[0][tid];
#pragma unroll
        for (int q = 1; q < 8; ++q) s = df_add(s, rb[q][tid]);
        const int64_t row = r0 + tid;
        const df64 x = row < dim ? df_sub(wr, s) : df_zero();
        if (PROJ) xs[tid] = x;
        if (row < dim) w[row] = x;
        dacc_fma(nacc, x, x);
      }
      if (PROJ) __syncthreads();
    }
    if (PROJ) {
      const float4 xv = UPD ? *reinterpret_cast<const float4*>(&xs[2 * lane]) : wv;
      const df64 x0 = make_df(xv.x, xv.y), x1 = make_df(xv.z, xv.w);
      if (!UPD && wp == 0) {
        dacc_fma(nacc, x0, x0);
        dacc_fma(nacc, x1, x1);
      }
#pragma unroll
      for (int m = 0; m < CPW; ++m) {
        if (m >= mycols) break;
        const float4 v = *reinterpret_cast<const float4*>(sl + 8 * m * LR);
        dacc_fma(acc[m], make_df(v.x, v.y), x0);
        dacc_fma(acc[m], make_df(v.z, v.w), x1);
      }
      if ((it & 15) == 15) {
#pragma unroll
        for (int m = 0; m < CPW; ++m) {
          if (m >= mycols) break;
          dacc_norm(acc[m]);
        }
      }
    }
    wr = wr_n;
    wv = wv_n;
  }
  cp_async_wait<0>();
  df64 nv = warp_sum_df(dacc_val(nacc));
  if (lane == 0) nred[wp] = nv;
  if (PROJ) {
#pragma unroll
    for (int m = 0; m < CPW; ++m) {
      if (m >= mycols) break;  // warp-uniform
      const df64 v = warp_sum_df(dacc_val(acc[m]));
      if (lane == 0) part[(int64_t)blockIdx.x * ldp + wp + 8 * m] = v;
    }
  }
  __syncthreads();
  if (tid == 0) {
    df64 t = nred[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) t = df_add(t, nred[q]);
    part[(int64_t)blockIdx.x * ldp + ncols] = t;
  }
}

}  // namespace ssa
