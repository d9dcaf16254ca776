// Reorthogonalisation against the Lanczos basis (section 3.2.2) by
// classical Gram-Schmidt: the tile-walking passes over the basis, their
// reductions with the Kahan-Parlett gate of the third pass, the wide-basis
// fallback passes, and the launcher.  All vectors are double-float (df64).
#include <mutex>
#include "lanczos.h"
#include "lanczos_dev.cuh"
#include "prof.h"

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

// Second-pass reduction: out[i] for i <= ncols (out[ncols] = ||w'||^2), and
// the Kahan-Parlett decision for the third pass: *gate = ||w'||^2 < ref/2
// with ref = ||w||^2 before the first update; without a third pass
// ||w'||^2 is the final squared norm.
__global__ void k_reduce_gate(const df64* __restrict__ part, int ntiles, int ldp, int ncols, df64* __restrict__ out,
                              const df64* __restrict__ ref, int* __restrict__ gate, df64* __restrict__ nrm) {
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

// Tile-walking CGS pass over Q (dim x ncols, ncols <= FUSED_MAXCOL):
//   UPD:  w <- w - Q h          (h read from memory)
//   PROJ: part[block][c] = sum over the block's tiles of Q[tile, c] . w[tile]
//   always: part[block][ncols] = sum of w.w over the block's tiles (after UPD)
// Persistent blocks walk tiles of FR rows; every thread copies its share of
// the next tile (all columns and the w rows) to shared memory with 16-byte
// asynchronous copies while the current tile is processed (double buffer).
// The compute threads read two rows at a time (128-bit shared loads) and
// accumulate with a 12-instruction double-float multiply-add.  (One-thread
// bulk copies of the 512-byte column segments measured slower: the copy
// engine serialises many small requests.)
constexpr int FR = 64;   // rows per tile
constexpr int FRP = 66;  // column stride in shared memory (16-byte aligned)
constexpr int NST = 2;   // pipeline stages (tiles in shared memory per block); 32-row tiles with
                         // 4 stages measured slower (more per-tile overhead)
template <bool UPD, bool PROJ>
__global__ void __launch_bounds__(256) k_cgs_tiles(const df64* __restrict__ Q, int64_t ldq, int ncols,
                                                   df64* __restrict__ w, int64_t dim, const df64* __restrict__ h,
                                                   df64* __restrict__ part, int ldp, int ntiles, const int* flag,
                                                   unsigned* status) {
  if (flag && *flag == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ df64 red[8];
  const int stage_elems = ncols * FRP + FR;
  df64* st0 = reinterpret_cast<df64*>(smem_raw);
  df64* hs = st0 + NST * stage_elems;
  const int tid = threadIdx.x;
  if (UPD)
    for (int c = tid; c < ncols; c += 256) hs[c] = h[c];
  auto issue = [&](int stg, int tile) {  // all threads: 16-byte asynchronous copies
    const int64_t r0 = (int64_t)tile * FR;
    df64* st = st0 + stg * stage_elems;
    for (int e = tid; e < (ncols + 1) * (FR / 2); e += 256) {
      const int c = e / (FR / 2), l = e - c * (FR / 2);
      const int64_t row = r0 + 2 * l;
      const bool ok = row < dim;
      if (c < ncols)
        cp_async16(st + c * FRP + 2 * l, ok ? (const void*)(Q + (int64_t)c * ldq + row) : (const void*)Q, ok);
      else
        cp_async16(st + ncols * FRP + 2 * l, ok ? (const void*)(w + row) : (const void*)w, ok);
    }
  };
  dacc acc0 = dacc_zero(), acc1 = dacc_zero();
  df64 nrm = df_zero();
  // prologue: the first NST-1 tiles of this block in flight
  for (int p = 0; p < NST - 1; ++p) {
    const int t = blockIdx.x + p * gridDim.x;
    if (t < ntiles) issue(p, t);
    cp_async_commit();
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int stage = it % NST;
    const int ahead = tile + (NST - 1) * gridDim.x;
    if (ahead < ntiles) issue((it + NST - 1) % NST, ahead);
    cp_async_commit();
    cp_async_wait<NST - 1>();
    __syncthreads();
    const df64* Qs = st0 + stage * stage_elems;
    df64* ws = const_cast<df64*>(Qs) + ncols * FRP;
    const int64_t r0 = (int64_t)tile * FR;
    {  // rows 2rp, 2rp+1 of w (updated when UPD); 8 threads per row pair split the columns
      const int rp = tid >> 3, q = tid & 7;
      dacc a0 = dacc_zero(), a1 = dacc_zero();
      if (UPD) {
        for (int c = q; c < ncols; c += 8) {
          const float4 v = *reinterpret_cast<const float4*>(Qs + c * FRP + 2 * rp);
          const df64 hc = hs[c];
          dacc_fma(a0, make_df(v.x, v.y), hc);
          dacc_fma(a1, make_df(v.z, v.w), hc);
        }
      }
      df64 s0 = dacc_val(a0), s1 = dacc_val(a1);
#pragma unroll
      for (int m = 1; m < 8; m <<= 1) {
        s0 = df_add(s0, shfl_xor_df(s0, m));
        s1 = df_add(s1, shfl_xor_df(s1, m));
      }
      __syncthreads();
      if (q == 0) {
        const int64_t g0 = r0 + 2 * rp;
        const df64 x0 = g0 < dim ? df_sub(ws[2 * rp], s0) : df_zero();
        const df64 x1 = g0 + 1 < dim ? df_sub(ws[2 * rp + 1], s1) : df_zero();
        ws[2 * rp] = x0;
        ws[2 * rp + 1] = x1;
        if (UPD) {
          if (g0 < dim) w[g0] = x0;
          if (g0 + 1 < dim) w[g0 + 1] = x1;
        }
        if (!PROJ) {
          nrm = df_fma(x0, x0, nrm);
          nrm = df_fma(x1, x1, nrm);
        }
      }
    }
    __syncthreads();
    if (PROJ) {  // two threads per column (one per half tile); column ncols is w.w
      const int half = tid & 1;
      const int c = tid >> 1, c1 = (tid + 256) >> 1;
      const float4* wv = reinterpret_cast<const float4*>(ws + half * (FR / 2));
      if (c <= ncols) {
        const float4* col = reinterpret_cast<const float4*>((c < ncols ? Qs + c * FRP : ws) + half * (FR / 2));
#pragma unroll 4
        for (int i = 0; i < FR / 4; ++i) {
          const float4 qv = col[i], xv = wv[i];
          dacc_fma(acc0, make_df(qv.x, qv.y), make_df(xv.x, xv.y));
          dacc_fma(acc0, make_df(qv.z, qv.w), make_df(xv.z, xv.w));
        }
        dacc_norm(acc0);
      }
      if (c1 <= ncols) {
        const float4* col = reinterpret_cast<const float4*>((c1 < ncols ? Qs + c1 * FRP : ws) + half * (FR / 2));
#pragma unroll 4
        for (int i = 0; i < FR / 4; ++i) {
          const float4 qv = col[i], xv = wv[i];
          dacc_fma(acc1, make_df(qv.x, qv.y), make_df(xv.x, xv.y));
          dacc_fma(acc1, make_df(qv.z, qv.w), make_df(xv.z, xv.w));
        }
        dacc_norm(acc1);
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  if (PROJ) {
    df64 v0 = dacc_val(acc0), v1 = dacc_val(acc1);
    v0 = df_add(v0, shfl_xor_df(v0, 1));
    v1 = df_add(v1, shfl_xor_df(v1, 1));
    const int c = tid >> 1, c1 = (tid + 256) >> 1;
    if ((tid & 1) == 0) {
      if (c <= ncols) part[(int64_t)blockIdx.x * ldp + c] = v0;
      if (c1 <= ncols) part[(int64_t)blockIdx.x * ldp + c1] = v1;
    }
  } else {
    nrm = warp_sum_df(nrm);
    if ((tid & 31) == 0) red[tid >> 5] = nrm;
    __syncthreads();
    if (tid == 0) {
      df64 t = df_zero();
      for (int i = 0; i < 8; ++i) t = df_add(t, red[i]);
      part[(int64_t)blockIdx.x * ldp + ncols] = t;
    }
  }
}

// out[0] = sum_b part[b][col] (one value), for the norm column
__global__ void k_reduce_one(const df64* __restrict__ part, int nblk, int ldp, int col, df64* __restrict__ out,
                             const int* flag) {
  if (flag && *flag == 0) return;
  df64 s = df_zero();
  for (int b = threadIdx.x; b < nblk; b += 32) s = df_add(s, part[(int64_t)b * ldp + col]);
  s = warp_sum_df(s);
  if (threadIdx.x == 0) *out = s;
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
int reorth_blocks(int64_t dim) { return (int)((dim + SLAB - 1) / SLAB); }
int fused_tiles(int64_t dim) { return (int)((dim + FR - 1) / FR); }
int fused_grid(size_t smem_bytes);

void launch_cgs2(const df64* Q, int64_t ldq, int ncols, df64* w, int64_t dim, ReorthWork& rw, int mode,
                 cudaStream_t s) {
  const int G = reorth_blocks(dim);
  // algorithmic bytes: the ncols basis columns once per pass, w read (and written by updates)
  const double qb = 8.0 * (double)dim * ncols;
  const double fl = 2.0 * (double)dim * ncols;
  const int* flag = nullptr;
  if (ncols <= FUSED_MAXCOL) {
    const int T2 = fused_tiles(dim);
    const size_t sm = ((size_t)NST * (ncols * FRP + FR) + ncols) * sizeof(df64);
    const int G2 = T2 < fused_grid(sm) ? T2 : fused_grid(sm);
    const int ldp = rw.ldp2;
    const df64* hlast = rw.h;
    const int* gate = nullptr;
    if (ncols > 0) {
      // pass 1: h = Q^T w and ||w||^2 (column ncols)
      prof_begin(s);
      k_cgs_tiles<false, true><<<G2, 256, sm, s>>>(Q, ldq, ncols, w, dim, rw.h, rw.part2, ldp, T2, flag, rw.status);
      prof_end(s, K_PROJ, qb + 8.0 * dim, fl);
      prof_begin(s);
      k_reduce_cols<<<(ncols + 8) / 8, 256, 0, s>>>(rw.part2, G2, ldp, ncols + 1, rw.h, flag);
      prof_end(s, K_MISC, 0.0, 0.0);
      if (mode == REORTH_GATED) {
        // pass 2: w <- w - Q h, h2 = Q^T w, ||w||^2; the gate decides on pass 3
        prof_begin(s);
        k_cgs_tiles<true, true><<<G2, 256, sm, s>>>(Q, ldq, ncols, w, dim, rw.h, rw.part2, ldp, T2, flag, rw.status);
        prof_end(s, K_UPDATE_PROJ, qb + 16.0 * dim, 2 * fl);
        prof_begin(s);
        k_reduce_gate<<<(ncols + 8) / 8, 256, 0, s>>>(rw.part2, G2, ldp, ncols, rw.h2, rw.h + ncols, rw.gate,
                                                      rw.nrm);
        prof_end(s, K_MISC, 0.0, 0.0);
        hlast = rw.h2;
        gate = rw.gate;
      }
    }
    // last pass: w <- w - Q h, ||w||^2 (skipped on the device when the gate is 0)
    prof_begin(s);
    k_cgs_tiles<true, false><<<G2, 256, sm, s>>>(Q, ldq, ncols, w, dim, hlast, rw.part2, ldp, T2, gate, rw.status);
    prof_end(s, gate ? K_GATED : K_UPDATE, gate ? 0.0 : qb + 16.0 * dim, gate ? 0.0 : fl);
    prof_begin(s);
    k_reduce_one<<<1, 32, 0, s>>>(rw.part2, G2, ldp, ncols, rw.nrm, gate);
    prof_end(s, K_MISC, 0.0, 0.0);
    return;
  }
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

// kernel attributes and the SM count, once per process (plans are created from many threads)
static std::once_flag g_reorth_once;
static int g_sms = 0;
void reorth_setup() {
  std::call_once(g_reorth_once, [] {
    const int mx = (int)(((size_t)NST * (FUSED_MAXCOL * FRP + FR) + FUSED_MAXCOL) * sizeof(df64));
    cudaFuncSetAttribute(k_cgs_tiles<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_cgs_tiles<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_cgs_tiles<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  });
}
// persistent grid of the fused pass: as many blocks as fit on every SM at once
int fused_grid(size_t smem_bytes) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cgs_tiles<true, true>, 256, smem_bytes);
  if (per < 1) per = 1;
  return (g_sms > 0 ? g_sms : 152) * per;
}

}  // namespace ssa
