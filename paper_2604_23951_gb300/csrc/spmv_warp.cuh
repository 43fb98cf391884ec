// Warp-tile engine for CSR SpMV with a fused per-row epilogue (sm_103a).
//
// Rows are sorted by length (longest first) and grouped into warp tiles of
// at most 32 consecutive rows.  Every warp of a persistent grid walks its
// tiles independently -- no CTA barrier inside the loop -- so the warps of an
// SM hide each other's memory latency.  In a tile each row is reduced by
// 2^v lanes, and each lane owns up to `nit` entries of its row per chunk (v
// and nit from the tile's longest row and the tile shape, so padding is
// bounded by the length spread inside one tile); a lane issues all its
// coalesced value / index loads and all its gathers of a chunk before its
// first multiply-add.  Group sums are combined with xor shuffles and moved
// to lane = row, so the epilogue runs with one lane per row.
//
// Rows too long for one warp's tile are either cut into segments (one warp
// each; the warp that completes a row's last segment adds the segments'
// partial sums in segment order and runs the row's epilogue) or, in the
// batched kernel, reduced by a whole CTA each.
//
// FP64 issue is scarce on GB300 (2 FP64 lanes per clock per SM), so the tile
// shape trades lanes per row (each costs a shuffle-add per pass) against
// chunks per lane (latency); the autotuner picks it per matrix.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace gb300lp {

constexpr int kWarpItems = 8;  // most entries one lane owns per chunk
constexpr int kCtaRow = 512;   // unsegmented plans: longer rows take one whole CTA each

// Where the epilogue of a segmented row leaves its accumulators: the check
// quantity q of long row r goes to p[q * stride + base + r] (a slot of its
// own, so the sums do not depend on which warp finished the row).
struct AccSink {
  double *p;
  int stride, base;
};

// Segmented rows of a matrix (tiles {r, INT_MIN | g}): row r's segments are
// seg_base[r] .. seg_base[r + 1] - 1, each of seg_len entries (the last one
// shorter); seg_part holds one partial sum per segment, seg_cnt one arrival
// counter per segmented row (zero between launches: the finishing warp
// resets it).  All NULL when the matrix has no segmented rows.
struct SegCtx {
  const int *seg_base;
  double *seg_part;
  int *seg_cnt;
  int seg_len;
  AccSink sink;
};

// ---- accumulators ---------------------------------------------------------
// Acc = double / float: plain multiply-adds.  Acc = F2: the mixed-precision
// SpMV, FP32 matrix values times a gathered vector held as a float pair
// hi + lo (split_f2: about 2^-48 relative), accumulated after the
// dot-product algorithm Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005): each product is split into its
// rounded value and its error (TwoProduct with an FMA; the lo part of the
// vector joins the error term), the running sum takes the rounded product
// through Knuth's TwoSum, and the error terms are summed on the side, so the
// result is about as accurate as a sum in twice FP32's precision of the
// products of the float-rounded matrix and the exact vector.  All of it runs
// on the FP32 pipe; the _rn intrinsics keep the compiler from fusing steps.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ float2 split_f2(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

template <typename Acc, typename T, typename V>
__device__ __forceinline__ void acc_mad(Acc &s, T a, V g) {
  s += (Acc)a * (Acc)g;
}
template <typename T>
__device__ __forceinline__ void acc_mad(F2 &s, T a_, float2 g) {
  const float a = (float)a_;
  const float p = __fmul_rn(a, g.x);
  // a * (g.x + g.y) - p: the FMA gives a * g.x - p exactly, plus a * g.y
  const float e = __fmaf_rn(a, g.y, __fmaf_rn(a, g.x, -p));
  const float t = __fadd_rn(s.hi, p);  // TwoSum: s.hi + p == t + q exactly
  const float z = __fsub_rn(t, s.hi);
  const float q = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(q, e));
}

template <typename Acc>
__device__ __forceinline__ void acc_add(Acc &s, Acc t) {
  s += t;
}
__device__ __forceinline__ void acc_add(F2 &s, F2 u) {
  const float t = __fadd_rn(s.hi, u.hi);
  const float z = __fsub_rn(t, s.hi);
  const float q = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(u.hi, z));
  s.hi = t;
  s.lo = __fadd_rn(__fadd_rn(s.lo, u.lo), q);
}

template <typename Acc>
__device__ __forceinline__ Acc acc_shfl_xor(Acc s, int o) {
  return __shfl_xor_sync(kFull, s, o);
}
__device__ __forceinline__ F2 acc_shfl_xor(F2 s, int o) {
  return F2{__shfl_xor_sync(kFull, s.hi, o), __shfl_xor_sync(kFull, s.lo, o)};
}
template <typename Acc>
__device__ __forceinline__ Acc acc_shfl(Acc s, int src) {
  return __shfl_sync(kFull, s, src);
}
__device__ __forceinline__ F2 acc_shfl(F2 s, int src) {
  return F2{__shfl_sync(kFull, s.hi, src), __shfl_sync(kFull, s.lo, src)};
}

template <typename Acc>
__device__ __forceinline__ double acc_value(Acc s) {
  return (double)s;
}
__device__ __forceinline__ double acc_value(F2 s) { return (double)s.hi + (double)s.lo; }

// A warp tile: rows [r0, r0 + nrows) with 2^vlog lanes per row and nit
// entries per lane per chunk, packed as int2 {r0, nrows | vlog << 8 |
// nit << 12}.
struct WarpTile {
  int r0, nrows, vlog, nit;
};

__host__ __device__ __forceinline__ int2 pack_wtile(int r0, int nrows, int vlog, int nit) {
  return make_int2(r0, nrows | (vlog << 8) | (nit << 12));
}

__device__ __forceinline__ WarpTile decode_wtile(int2 v) {
  WarpTile w;
  w.r0 = v.x;
  w.nrows = v.y & 0xff;
  w.vlog = (v.y >> 8) & 0xf;
  w.nit = v.y >> 12;
  return w;
}

// sum over the entries lo + gl, lo + gl + vl, ... < hi of va[k] * vec[ci[k]],
// NIT entries per chunk: all loads and gathers of a chunk before its FMAs
template <int NIT, typename T, typename V, typename Acc>
__device__ __forceinline__ Acc group_dot(int lo, int hi, int gl, int vl,
                                         const int *__restrict__ ci, const T *__restrict__ va,
                                         const V *__restrict__ vec) {
  Acc s{};
  const int span = vl * NIT;
  for (int k0 = lo + gl; k0 < hi; k0 += span) {
    int j[NIT];
    T a[NIT];
#pragma unroll
    for (int u = 0; u < NIT; ++u) {
      const int k = k0 + u * vl;
      j[u] = k < hi ? ci[k] : 0;
      a[u] = k < hi ? va[k] : (T)0;
    }
    V g[NIT];
#pragma unroll
    for (int u = 0; u < NIT; ++u) g[u] = vec[j[u]];
#pragma unroll
    for (int u = 0; u < NIT; ++u) acc_mad(s, a[u], g[u]);
  }
  return s;
}

// Rows [0, nlong), one per CTA (cta, cta + ncta, ...), each reduced by the
// whole CTA (entries per thread sized to the row, at most kWarpItems per
// chunk); epi.pre / epi.row run on thread 0.
template <typename T, typename V, typename Acc, class Epi>
__device__ __forceinline__ void cta_rows(int nlong, const int *__restrict__ rp,
                                         const int *__restrict__ ci, const T *__restrict__ va,
                                         const V *__restrict__ vec, Epi &epi, Acc *red, int cta,
                                         int ncta) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nthr = blockDim.x;
  const int nwarp = nthr >> 5;
  for (int r = cta; r < nlong; r += ncta) {
    if (threadIdx.x == 0) epi.pre(r);
    const int lo = rp[r], hi = rp[r + 1];
    // entries per thread per chunk: just enough for one chunk, at most
    // kWarpItems (CTA-uniform)
    const int nit = min(kWarpItems, max(1, (hi - lo + nthr - 1) / nthr));
    Acc s{};
    switch (nit) {
      case 1: s = group_dot<1, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      case 2: s = group_dot<2, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      case 3: s = group_dot<3, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      case 4: s = group_dot<4, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      case 5: s = group_dot<5, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      case 6: s = group_dot<6, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      case 7: s = group_dot<7, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
      default: s = group_dot<8, T, V, Acc>(lo, hi, threadIdx.x, nthr, ci, va, vec); break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_add(s, acc_shfl_xor(s, o));
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      Acc t{};
      for (int w = 0; w < nwarp; ++w) acc_add(t, red[w]);
      epi.row(r, acc_value(t));
    }
    __syncthreads();
  }
}

// The work is shared by ncta CTAs (this one is number cta): rows [0, nlong)
// (longer than kCtaRow) are reduced one per CTA (cta, cta + ncta, ...) by the
// whole CTA; then each warp walks its warp tiles (wid, wid + wstride, ...).  For
// every row r: epi.pre(r) then epi.row(r, sum_k va[k] * vec[ci[k]]), both on
// the same thread.  red: blockDim.x / 32 Acc of shared memory.
// One segment g of segmented row r (a whole warp): its partial sum goes to
// seg_part[g]; the warp whose arrival completes the row adds the row's
// partials in segment order (a fixed shuffle tree: the result does not depend
// on the arrival order), resets the row's counter and runs the epilogue on a
// copy of `epi` whose accumulators go to the row's own slots in sc.sink.
// No warp waits for another.
template <typename T, typename V, typename Acc, class Epi>
__device__ __forceinline__ void segment_tile(int r, int g, const int *__restrict__ rp,
                                             const int *__restrict__ ci,
                                             const T *__restrict__ va,
                                             const V *__restrict__ vec, const Epi &epi,
                                             const SegCtx &sc) {
  const int lane = threadIdx.x & 31;
  const int sb = sc.seg_base[r];
  const int nseg = sc.seg_base[r + 1] - sb;
  const int lo = rp[r] + (g - sb) * sc.seg_len;
  const int hi = min(lo + sc.seg_len, rp[r + 1]);
  Acc s = group_dot<kWarpItems, T, V, Acc>(lo, hi, lane, 32, ci, va, vec);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc_add(s, acc_shfl_xor(s, o));
  int last = 0;
  if (lane == 0) {
    sc.seg_part[g] = acc_value(s);
    __threadfence();
    last = atomicAdd(&sc.seg_cnt[r], 1) == nseg - 1;
  }
  last = __shfl_sync(kFull, last, 0);
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int q = lane; q < nseg; q += 32) t += __ldcg(&sc.seg_part[sb + q]);
  t = warp_sum(t);
  if (lane == 0) {
    sc.seg_cnt[r] = 0;
    Epi e = epi;
    e.clear();
    e.pre(r);
    e.row(r, t);
    e.sink(sc.sink, r);
  }
}

template <typename T, typename V, typename Acc, class Epi>
__device__ __forceinline__ void warp_spmv(int nlong, const int2 *__restrict__ tiles, int ntiles,
                                          const int *__restrict__ rp, const int *__restrict__ ci,
                                          const T *__restrict__ va, const V *__restrict__ vec,
                                          Epi &epi, Acc *red, int cta, int ncta,
                                          const SegCtx &sc = SegCtx{}) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nthr = blockDim.x;
  const int nwarp = nthr >> 5;
  cta_rows<T, V, Acc>(nlong, rp, ci, va, vec, epi, red, cta, ncta);
  // ---- warp tiles ---------------------------------------------------------
  const int wid = cta * nwarp + warp;
  const int wstride = ncta * nwarp;
  for (int t = wid; t < ntiles; t += wstride) {
    const int2 raw = tiles[t];
    if (raw.y < 0) {
      segment_tile<T, V, Acc>(raw.x, raw.y & 0x7fffffff, rp, ci, va, vec, epi, sc);
      continue;
    }
    const WarpTile w = decode_wtile(raw);
    const bool has = lane < w.nrows;
    if (has) epi.pre(w.r0 + lane);
    // row offsets of the tile, one row per lane
    const int my_lo = has ? rp[w.r0 + lane] : 0;
    const int my_hi = has ? rp[w.r0 + lane + 1] : 0;
    Acc mine{};
    const int vlog = w.vlog;
    const int vl = 1 << vlog;
    const int rpp = 32 >> vlog;  // rows per pass
    const int g = lane >> vlog, gl = lane & (vl - 1);
    for (int p0 = 0; p0 < w.nrows; p0 += rpp) {
      const int q = p0 + g;  // row of this lane's group (may be past the tile)
      const int lo = __shfl_sync(kFull, my_lo, q & 31);
      const int hi = __shfl_sync(kFull, my_hi, q & 31);
      Acc s{};
      if (q < w.nrows) {
        switch (w.nit) {
          case 1: s = group_dot<1, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          case 2: s = group_dot<2, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          case 3: s = group_dot<3, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          case 4: s = group_dot<4, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          case 5: s = group_dot<5, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          case 6: s = group_dot<6, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          case 7: s = group_dot<7, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
          default: s = group_dot<8, T, V, Acc>(lo, hi, gl, vl, ci, va, vec); break;
        }
      }
      for (int o = vl >> 1; o > 0; o >>= 1) acc_add(s, acc_shfl_xor(s, o));
      // lane L keeps the sum of row L when row L was reduced in this pass
      const int src = ((lane - p0) & (rpp - 1)) << vlog;
      const Acc got = acc_shfl(s, src);
      if (lane >= p0 && lane < p0 + rpp) mine = got;
    }
    if (has) epi.row(w.r0 + lane, acc_value(mine));
  }
}

}  // namespace gb300lp
