// Warp-tile engine for CSR SpMV with a fused per-row epilogue (sm_103a).
//
// Rows are sorted by length (longest first) and grouped into warp tiles of
// at most 32 consecutive rows.  Every warp of a persistent grid walks its
// tiles independently -- no CTA barrier inside the loop -- so the warps of an
// SM hide each other's memory latency.  In a tile each row is reduced by
// 2^v lanes (v from the tile's longest row, so no lane owns more than
// kWarpItems entries); a lane issues all its coalesced value / index loads
// and all its gathers before its first multiply-add.  Group sums are
// combined with xor shuffles and moved to lane = row, so the epilogue runs
// with one lane per row and all lanes active.  A warp tile holds about
// kWarpTileNnz nonzeros so the tiles balance across warps; rows longer than
// 32 * kWarpItems come first and are each reduced by a whole CTA.
//
// FP64 issue is scarce on GB300 (2 FP64 lanes per clock per SM): the
// length-sorted tiles keep the multiply-adds at full lanes and the epilogue
// never runs with idle lanes.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace gb300lp {

#ifndef GB300_WARP_ITEMS
#define GB300_WARP_ITEMS 8
#endif
constexpr int kWarpItems = GB300_WARP_ITEMS;  // entries one lane owns per pass
constexpr int kLongRow = 32 * kWarpItems;      // longer rows: single-row tiles

constexpr int kWarpTileNnz = 512;             // nonzeros a warp tile aims at

// A warp tile: rows [r0, r0 + nrows) with lanes per row 2^vlog, packed as
// int2 {r0, nrows | vlog << 8}.  Rows longer than kLongRow are not in warp
// tiles: they come first in the row order and each is reduced by a whole CTA.
constexpr int kWarpLongMode = 6;

struct WarpTile {
  int r0, nrows, vlog;
};

__device__ __forceinline__ WarpTile load_wtile(const int2 *__restrict__ tiles, int t) {
  int2 v = tiles[t];
  WarpTile w;
  w.r0 = v.x;
  w.nrows = v.y & 0xff;
  w.vlog = v.y >> 8;
  return w;
}

// The work is shared by ncta CTAs (this one is number cta): rows [0, nlong)
// are long rows, one per CTA (cta, cta + ncta, ...), reduced by the whole
// CTA; then each warp walks its warp tiles (wid, wid + wstride, ...).  For
// every row r: epi.pre(r) then epi.row(r, sum_k va[k] * vec[ci[k]]), both on
// the same thread.  red: blockDim.x / 32 Acc of shared memory.
template <typename T, typename V, typename Acc, class Epi>
__device__ __forceinline__ void warp_spmv(int nlong, const int2 *__restrict__ tiles, int ntiles,
                                          const int *__restrict__ rp, const int *__restrict__ ci,
                                          const T *__restrict__ va, const V *__restrict__ vec,
                                          Epi &epi, Acc *red, int cta, int ncta) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nthr = blockDim.x;
  const int nwarp = nthr >> 5;
  // ---- long rows: whole CTA per row ------------------------------------
  for (int r = cta; r < nlong; r += ncta) {
    if (threadIdx.x == 0) epi.pre(r);
    const int lo = rp[r], hi = rp[r + 1];
    Acc s = 0;
    for (int base = lo + threadIdx.x; base < hi; base += nthr * kWarpItems) {
      int j[kWarpItems];
      T a[kWarpItems];
#pragma unroll
      for (int u = 0; u < kWarpItems; ++u) {
        const int k = base + nthr * u;
        j[u] = k < hi ? ci[k] : 0;
        a[u] = k < hi ? va[k] : (T)0;
      }
      V g[kWarpItems];
#pragma unroll
      for (int u = 0; u < kWarpItems; ++u) g[u] = vec[j[u]];
#pragma unroll
      for (int u = 0; u < kWarpItems; ++u) s += (Acc)a[u] * (Acc)g[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      Acc t = 0;
      for (int w = 0; w < nwarp; ++w) t += red[w];
      epi.row(r, (double)t);
    }
    __syncthreads();
  }
  // ---- warp tiles ---------------------------------------------------------
  const int wid = cta * nwarp + warp;
  const int wstride = ncta * nwarp;
  for (int t = wid; t < ntiles; t += wstride) {
    const WarpTile w = load_wtile(tiles, t);
    const bool has = lane < w.nrows;
    if (has) epi.pre(w.r0 + lane);
    // row offsets of the tile, one row per lane
    const int my_lo = has ? rp[w.r0 + lane] : 0;
    const int my_hi = has ? rp[w.r0 + lane + 1] : 0;
    Acc mine = 0;
    const int vlog = w.vlog;
    const int vl = 1 << vlog;
    const int rpp = 32 >> vlog;  // rows per pass
    const int g = lane >> vlog, gl = lane & (vl - 1);
    for (int p0 = 0; p0 < w.nrows; p0 += rpp) {
      const int q = p0 + g;  // row of this lane's group (may be past the tile)
      const int lo = __shfl_sync(kFull, my_lo, q & 31);
      const int hi = __shfl_sync(kFull, my_hi, q & 31);
      Acc s = 0;
      if (q < w.nrows) {
        int j[kWarpItems];
        T a[kWarpItems];
#pragma unroll
        for (int u = 0; u < kWarpItems; ++u) {
          const int k = lo + gl + u * vl;
          j[u] = k < hi ? ci[k] : 0;
          a[u] = k < hi ? va[k] : (T)0;
        }
        V gv[kWarpItems];
#pragma unroll
        for (int u = 0; u < kWarpItems; ++u) gv[u] = vec[j[u]];
#pragma unroll
        for (int u = 0; u < kWarpItems; ++u) s += (Acc)a[u] * (Acc)gv[u];
      }
      for (int o = vl >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
      // lane L keeps the sum of row L when row L was reduced in this pass
      const int src = ((lane - p0) & (rpp - 1)) << vlog;
      const Acc got = __shfl_sync(kFull, s, src);
      if (lane >= p0 && lane < p0 + rpp) mine = got;
    }
    if (has) epi.row(w.r0 + lane, (double)mine);
  }
}

}  // namespace gb300lp
