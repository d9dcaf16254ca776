// Reorthogonalisation against the Lanczos basis (section 3.2.2) by
// classical Gram-Schmidt: the launcher of the fused lane-owned passes (the
// kernel is in cgs_lanes.cuh), their reductions with the Kahan-Parlett gate
// of the third pass, and the wide-basis fallback passes.  All vectors are
// double-float (df64).
#include <mutex>
#include "lanczos.h"
#include "lanczos_dev.cuh"
#include "prof.h"
#include "cgs_lanes.cuh"

namespace ssa {


// ---------------------------------------------------------------- CGS pieces
// Bases wider than FUSED_MAXCOL: two projection/update rounds as separate
// passes over the basis Q (dim x ncols, column-major):
//   h = Q^T w (k_cgs_proj, partial sums per row tile, reduced by
//   k_reduce_cols in tile order), then w <- w - Q h and ||w||^2 (k_cgs_update).

// P1: part[tile][i] = sum over the tile's rows of Q[:, i] w for i < ncols,
// and part[tile][ncols] = w.w.  Columns go in batches of 4 so each thread has
// 16 independent 16-byte loads in flight.
__global__ void __launch_bounds__(RT) k_cgs_proj(const df64* __restrict__ Q, int64_t ldq, int ncols,
                                                 const df64* __restrict__ w, int64_t dim, df64* __restrict__ part,
                                                 int ldp, const int* flag) {
  if (flag && *flag == 0) return;
  __shared__ df64 red[RT / 32][MAXCOL + 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * SLAB;
  df64 wv[RP][2];
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
    float4 v = ld_pair(w, row, dim);
    wv[p][0] = make_df(v.x, v.y);
    wv[p][1] = make_df(v.z, v.w);
  }
  for (int c0 = 0; c0 <= ncols; c0 += 4) {
    float4 q[4][RP];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int col = c0 + b;
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
        if (col < ncols) q[b][p] = ld_pair(Q + (int64_t)col * ldq, row, dim);
        else if (col == ncols) q[b][p] = make_float4(wv[p][0].hi, wv[p][0].lo, wv[p][1].hi, wv[p][1].lo);
        else q[b][p] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    df64 acc[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[b] = df_zero();
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        acc[b] = df_fma(make_df(q[b][p].x, q[b][p].y), wv[p][0], acc[b]);
        acc[b] = df_fma(make_df(q[b][p].z, q[b][p].w), wv[p][1], acc[b]);
      }
    }
    const df64 u = warp_sum4_df(acc[0], acc[1], acc[2], acc[3]);
    if ((lane & 7) == 0) red[warp][c0 + (lane >> 3)] = u;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= ncols; i += RT) {
    df64 s = df_zero();
#pragma unroll
    for (int wp = 0; wp < RT / 32; ++wp) s = df_add(s, red[wp][i]);
    part[(int64_t)blockIdx.x * ldp + i] = s;
  }
}

// out[i] = sum_t part[t][i] for i < ncols (tile order, one warp per column)
__global__ void k_reduce_cols(const df64* __restrict__ part, int ntiles, int ldp, int ncols, df64* __restrict__ out,
                              const int* flag) {
  if (flag && *flag == 0) return;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  df64 s = df_zero();
  for (int t = lane; t < ntiles; t += 32) s = df_add(s, part[(int64_t)t * ldp + col]);
  s = warp_sum_df(s);
  if (lane == 0) out[col] = s;
}

// First-pass reduction with the skip test ("orthogonalise only when
// necessary", section 3.2.2, with the loss measured instead of estimated):
// out[i] = sum_t part[t][i] for i <= ncols (out[ncols] = ||w||^2).  The
// product w is not reduced by the recurrence term beforehand, so its
// coefficient on the newest column, h_l (l = ncols - 1), is the coupling of
// the bidiagonalisation and is always large; with w' = w - h_l q_l
// (||w'||^2 ~ ||w||^2 - h_l^2), the last block skips the rest of the
// Gram-Schmidt when
//   max_{i<l} |h_i| <= tau ||w'||   (w' already orthogonal to the older columns)
//   ||w||^2 <= SKIP_RATIO ||w'||^2   (one projection on q_l leaves at most
//                                     ~1e-14 ||w|| / ||w'|| along it)
// Then *run = 0 (no update + second projection), *gate = 0 (no third pass)
// and *skip = 1: the normalisation forms w' itself.  Otherwise *run = 1,
// *skip = 0.
__global__ void k_reduce_skip(const df64* __restrict__ part, int ntiles, int ldp, int ncols, df64* __restrict__ out,
                              int* __restrict__ run, int* __restrict__ gate, int* __restrict__ skip, double tau,
                              int* __restrict__ counter) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col <= ncols) {
    df64 s = df_zero();
    for (int t = lane; t < ntiles; t += 32) s = df_add(s, part[(int64_t)t * ldp + col]);
    s = warp_sum_df(s);
    if (lane == 0) out[col] = s;
  }
  if (!last_block(counter)) return;
  __shared__ float wmax[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < ncols - 1; i += blockDim.x) {
    const volatile df64* hp = out + i;
    m = fmaxf(m, fabsf(hp->hi));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, wmax[i]);
    const volatile df64* wp = out + ncols;
    const volatile df64* lp = out + (ncols - 1);
    const double w2 = df_to_double(make_df(wp->hi, wp->lo));
    const double hl = df_to_double(make_df(lp->hi, lp->lo));
    const double r2 = w2 - hl * hl;  // ||w'||^2, good to a few digits when the ratio test passes
    const double hm = (double)m;
    const bool skipped = ncols >= 1 && r2 > 0.0 && hm * hm <= tau * tau * r2 && w2 <= SKIP_RATIO * r2;
    *run = skipped ? 0 : 1;
    *skip = skipped ? 1 : 0;
    if (skipped) *gate = 0;
    *counter = 0;
  }
}

// Second-pass reduction: out[i] for i <= ncols (out[ncols] = ||w'||^2), and
// the Kahan-Parlett decision for the third pass: *gate = ||w'||^2 < ref/2
// with ref = ||w||^2 before the first update; without a third pass
// ||w'||^2 is the final squared norm.
__global__ void k_reduce_gate(const df64* __restrict__ part, int ntiles, int ldp, int ncols, df64* __restrict__ out,
                              const df64* __restrict__ ref, int* __restrict__ gate, df64* __restrict__ nrm,
                              const int* flag) {
  if (flag && *flag == 0) return;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col > ncols) return;
  df64 s = df_zero();
  for (int t = lane; t < ntiles; t += 32) s = df_add(s, part[(int64_t)t * ldp + col]);
  s = warp_sum_df(s);
  if (lane == 0) {
    out[col] = s;
    if (col == ncols) {
      const bool again = df_lt(df_scale(s, 2.0f), *ref);
      *gate = again ? 1 : 0;
      if (!again) *nrm = s;
    }
  }
}

// P3: w -= Q h; part[tile] = w.w over the tile; the last block sums the
// tile partials into *nrm_out.  Columns in batches of 4 for load parallelism.
__global__ void __launch_bounds__(RT) k_cgs_update(const df64* __restrict__ Q, int64_t ldq, int ncols,
                                                   df64* __restrict__ w, int64_t dim, const df64* __restrict__ h,
                                                   df64* __restrict__ part, df64* __restrict__ nrm_out,
                                                   int* counter, const int* flag) {
  if (flag && *flag == 0) return;
  __shared__ df64 hs[MAXCOL + 4];
  __shared__ df64 red[RT / 32];
  for (int i = threadIdx.x; i < ncols; i += RT) hs[i] = h[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * SLAB;
  df64 acc[RP][2];
#pragma unroll
  for (int p = 0; p < RP; ++p) acc[p][0] = acc[p][1] = df_zero();
  int c0 = 0;
  for (; c0 + 4 <= ncols; c0 += 4) {
    float4 q[4][RP];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int p = 0; p < RP; ++p)
        q[b][p] = ld_pair(Q + (int64_t)(c0 + b) * ldq, r0 + 2 * ((int64_t)threadIdx.x + p * RT), dim);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const df64 hb = hs[c0 + b];
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        acc[p][0] = df_fma(make_df(q[b][p].x, q[b][p].y), hb, acc[p][0]);
        acc[p][1] = df_fma(make_df(q[b][p].z, q[b][p].w), hb, acc[p][1]);
      }
    }
  }
  for (; c0 < ncols; ++c0) {
    const df64 hb = hs[c0];
#pragma unroll
    for (int p = 0; p < RP; ++p) {
      const float4 v = ld_pair(Q + (int64_t)c0 * ldq, r0 + 2 * ((int64_t)threadIdx.x + p * RT), dim);
      acc[p][0] = df_fma(make_df(v.x, v.y), hb, acc[p][0]);
      acc[p][1] = df_fma(make_df(v.z, v.w), hb, acc[p][1]);
    }
  }
  df64 nrm = df_zero();
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    const int64_t row = r0 + 2 * ((int64_t)threadIdx.x + p * RT);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (row + e < dim) {
        df64 x = df_sub(w[row + e], acc[p][e]);
        w[row + e] = x;
        nrm = df_fma(x, x, nrm);
      }
    }
  }
  nrm = warp_sum_df(nrm);
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    df64 s = df_zero();
    for (int wp = 0; wp < RT / 32; ++wp) s = df_add(s, red[wp]);
    part[blockIdx.x] = s;
  }
  if (last_block(counter)) {
    if (threadIdx.x == 0) {
      df64 s = df_zero();
      for (int b = 0; b < (int)gridDim.x; ++b) {
        const volatile df64* pp = part + b;
        s = df_add(s, make_df(pp->hi, pp->lo));
      }
      *nrm_out = s;
      *counter = 0;
    }
  }
}


// ---------------------------------------------------------------- launchers
// While launch statistics are on, a pass that the device may skip is charged
// to its class with its bytes only if it runs: the flag is read back first
// (a synchronisation outside the timed launches).  Without statistics the
// decision stays on the device.
static bool flag_on_host(const int* flag, cudaStream_t s) {
  if (!prof_enabled() || !flag) return true;
  int v = 1;
  if (cudaMemcpyAsync(&v, flag, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return true;
  return v != 0;
}

constexpr int LNST = 2;  // staged tiles per block: two blocks per SM fit bases up to ~104 columns
int reorth_blocks(int64_t dim) { return (int)((dim + SLAB - 1) / SLAB); }
int fused_tiles(int64_t dim) { return (int)((dim + LR - 1) / LR); }

// persistent grid of the fused passes per [pass][ncols]: as many blocks as fit on every SM at once
enum { P_PROJ = 0, P_UPD_PROJ = 1, P_UPD = 2 };
static int g_lanes_grid[3][FUSED_MAXCOL + 1];
static int g_sms = 0;

template <bool UPD, bool PROJ, int CPW>
static void lanes_one(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, const df64* h, df64* part,
                      int ldp, int G, int T, const int* flag, cudaStream_t s) {
  const size_t sm = (size_t)LNST * ncols * LR * sizeof(df64);
  k_cgs_lanes<UPD, PROJ, CPW, LNST><<<G, 256, sm, s>>>(Q, ldq, ncols, w, dim, h, part, ldp, T, flag);
}
template <bool UPD, bool PROJ>
static void lanes_pass(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, const df64* h, df64* part,
                       int ldp, int G, int T, const int* flag, cudaStream_t s) {
  if (ncols <= 32) lanes_one<UPD, PROJ, 4>(Q, ldq, ncols, w, dim, h, part, ldp, G, T, flag, s);
  else if (ncols <= 64) lanes_one<UPD, PROJ, 8>(Q, ldq, ncols, w, dim, h, part, ldp, G, T, flag, s);
  else if (ncols <= 104) lanes_one<UPD, PROJ, 13>(Q, ldq, ncols, w, dim, h, part, ldp, G, T, flag, s);
  else lanes_one<UPD, PROJ, 25>(Q, ldq, ncols, w, dim, h, part, ldp, G, T, flag, s);
}

void launch_cgs2(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, ReorthWork& rw, int mode,
                 cudaStream_t s) {
  const int G = reorth_blocks(dim);
  // algorithmic bytes: the ncols basis columns once per pass, w read (and written by updates)
  const double qb = 8.0 * (double)dim * ncols;
  const double fl = 2.0 * (double)dim * ncols;
  // REORTH_PRO: every pass waits on the partial-reorthogonalisation decision
  const int* flag = mode == REORTH_PRO ? rw.run : nullptr;
  const bool gated = mode == REORTH_GATED || mode == REORTH_PRO;
  if (ncols <= FUSED_MAXCOL) {
    const int T2 = fused_tiles(dim);
    auto grid = [&](int pass) {
      int g = g_lanes_grid[pass][ncols] < T2 ? g_lanes_grid[pass][ncols] : T2;
      return rw.grid_cap > 0 && g > rw.grid_cap ? rw.grid_cap : g;
    };
    const int ldp = rw.ldp2;
    const df64* hlast = rw.h;
    const int* gate = nullptr;
    if (ncols > 0) {
      // pass 1: h = Q^T w and ||w||^2 (column ncols)
      const int G1 = grid(P_PROJ);
      const bool ran1 = flag_on_host(flag, s);
      prof_begin(s);
      lanes_pass<false, true>(Q, ldq, ncols, w, dim, rw.h, rw.part2, ldp, G1, T2, flag, s);
      prof_end(s, ran1 ? K_PROJ : K_SKIPPED, ran1 ? qb + 8.0 * dim : 0.0, ran1 ? fl : 0.0);
      if (gated) {
        const bool skip_test = mode == REORTH_GATED && rw.skip_tau > 0.0;
        const int* run = skip_test || mode == REORTH_PRO ? rw.run : nullptr;
        prof_begin(s);
        if (skip_test)  // the skip test decides on the device whether passes 2 and 3 run
          k_reduce_skip<<<(ncols + 8) / 8, 256, 0, s>>>(rw.part2, G1, ldp, ncols, rw.h, rw.run, rw.gate, rw.skip,
                                                        rw.skip_tau, rw.counter);
        else
          k_reduce_cols<<<(ncols + 8) / 8, 256, 0, s>>>(rw.part2, G1, ldp, ncols + 1, rw.h, flag);
        prof_end(s, K_MISC, 0.0, 0.0);
        // pass 2: w <- w - Q h, h2 = Q^T w, ||w||^2; the gate decides on pass 3
        const int G2 = grid(P_UPD_PROJ);
        const bool ran2 = flag_on_host(run, s);
        prof_begin(s);
        lanes_pass<true, true>(Q, ldq, ncols, w, dim, rw.h, rw.part2, ldp, G2, T2, run, s);
        prof_end(s, ran2 ? K_UPDATE_PROJ : K_SKIPPED, ran2 ? qb + 16.0 * dim : 0.0, ran2 ? 2 * fl : 0.0);
        prof_begin(s);
        k_reduce_gate<<<(ncols + 8) / 8, 256, 0, s>>>(rw.part2, G2, ldp, ncols, rw.h2, rw.h + ncols, rw.gate,
                                                      rw.nrm, run);
        prof_end(s, K_MISC, 0.0, 0.0);
        hlast = rw.h2;
        gate = rw.gate;
      } else {
        prof_begin(s);
        k_reduce_cols<<<(ncols + 8) / 8, 256, 0, s>>>(rw.part2, G1, ldp, ncols + 1, rw.h, flag);
        prof_end(s, K_MISC, 0.0, 0.0);
      }
    }
    // last pass: w <- w - Q h, ||w||^2 (skipped on the device when the gate is 0)
    const int G3 = grid(P_UPD);
    const bool ran3 = gate ? flag_on_host(gate, s) : true;
    prof_begin(s);
    lanes_pass<true, false>(Q, ldq, ncols, w, dim, hlast, rw.part2, ldp, G3, T2, gate, s);
    prof_end(s, ran3 ? K_UPDATE : K_SKIPPED, ran3 ? qb + 16.0 * dim : 0.0, ran3 ? fl : 0.0);
    // the normalisation adds up the last pass's partial norms (unless the gate skipped that pass),
    // or, when the skip test fired, forms w - h_l q_l and its norm itself
    rw.nrm_blocks = G3;
    rw.nrm_col = ncols;
    rw.nrm_gate = gate;
    rw.skip_flag = (mode == REORTH_GATED && ncols > 0 && rw.skip_tau > 0.0) ? rw.skip : nullptr;
    return;
  }
  rw.nrm_blocks = 0;
  rw.skip_flag = nullptr;
  // wide bases: batched passes (four reads of Q)
  prof_begin(s);
  k_cgs_proj<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.part, rw.ldp, flag);
  prof_end(s, K_PROJ, qb + 8.0 * dim, fl);
  prof_begin(s);
  k_reduce_cols<<<(ncols + 7) / 8, 256, 0, s>>>(rw.part, G, rw.ldp, ncols, rw.h, flag);
  prof_end(s, K_MISC, 0.0, 0.0);
  prof_begin(s);
  k_cgs_update<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.h, rw.part, rw.nrm, rw.counter, flag);
  prof_end(s, K_UPDATE, qb + 16.0 * dim, fl);
  prof_begin(s);
  k_cgs_proj<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.part, rw.ldp, flag);
  prof_end(s, K_PROJ, qb + 8.0 * dim, fl);
  prof_begin(s);
  k_reduce_cols<<<(ncols + 7) / 8, 256, 0, s>>>(rw.part, G, rw.ldp, ncols, rw.h, flag);
  prof_end(s, K_MISC, 0.0, 0.0);
  prof_begin(s);
  k_cgs_update<<<G, RT, 0, s>>>(Q, ldq, ncols, w, dim, rw.h, rw.part, rw.nrm, rw.counter, flag);
  prof_end(s, K_UPDATE, qb + 16.0 * dim, fl);
}

// kernel attributes, the SM count and the grid table, once per process (plans are created
// from many threads)
template <bool UPD, bool PROJ, int CPW>
static void lanes_setup_one(int pass, int lo, int hi) {
  auto fn = k_cgs_lanes<UPD, PROJ, CPW, LNST>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(LNST * 8 * CPW * LR * sizeof(df64)));
  for (int n = lo; n <= hi; ++n) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, (size_t)LNST * n * LR * sizeof(df64));
    g_lanes_grid[pass][n] = (g_sms > 0 ? g_sms : 152) * (per < 1 ? 1 : per);
  }
}
template <bool UPD, bool PROJ>
static void lanes_setup(int pass) {
  lanes_setup_one<UPD, PROJ, 4>(pass, 0, 32);
  lanes_setup_one<UPD, PROJ, 8>(pass, 33, 64);
  lanes_setup_one<UPD, PROJ, 13>(pass, 65, 104);
  lanes_setup_one<UPD, PROJ, 25>(pass, 105, FUSED_MAXCOL);
}
static_assert(FUSED_MAXCOL <= 8 * 25, "fused passes hold at most 25 columns per warp");
static std::once_flag g_reorth_once;
void reorth_setup() {
  std::call_once(g_reorth_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    lanes_setup<false, true>(P_PROJ);
    lanes_setup<true, true>(P_UPD_PROJ);
    lanes_setup<true, false>(P_UPD);
  });
}

}  // namespace ssa
