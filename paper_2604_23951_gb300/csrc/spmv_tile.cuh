// Tile engine for CSR SpMV with a fused per-row epilogue (sm_103a).
//
// The rows of a matrix are sorted by length and cut into tiles of at most
// kTileRows consecutive rows and kTileNnz nonzeros.  A persistent CTA walks
// its tiles; for each tile one thread issues TMA bulk copies
// (cp.async.bulk, completion on an mbarrier) of the tile's contiguous
// values and column indices into shared memory, double buffered so the next
// tile streams in while the current one is reduced.  Row sums are formed
// from shared memory (one thread per row for short rows, a warp per row for
// medium rows, the whole CTA for rows of hundreds of entries), parked in
// shared memory, and the epilogue then runs with one thread per row and all
// lanes active.  Rows longer than kTileNnz form single-row tiles reduced by
// the whole CTA straight from global memory.
//
// FP64 arithmetic is scarce on GB300 (about 2 lanes per clock per SM), so
// the layout aims at full-lane FP64 instructions: length-sorted rows make
// thread-per-row loops nearly divergence free, and the epilogue never runs
// with idle lanes.
//
// Every wait on an mbarrier is bounded; on expiry the CTA records an error
// code in *err, waits (bounded) for its own copies in flight and returns.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace gb300lp {

constexpr int kTB = 256;        // threads per CTA
constexpr int kTileRows = 256;  // rows per tile (one epilogue thread each)
constexpr int kTileNnz = 2048;  // nonzeros per staged tile
constexpr int kTilePad = 8;     // alignment slack of a staged range

// tile modes (bits 29..31 of the packed row end)
enum TileMode { TM_THREAD = 0, TM_WARP = 1, TM_BLOCK = 2, TM_LONG = 3 };
constexpr int kModeShift = 29;
constexpr int kRowMask = (1 << kModeShift) - 1;

// 16-byte aligned staging area for one tile
template <typename T>
struct alignas(16) TileBuf {
  T val[kTileNnz + kTilePad];
  int ci[kTileNnz + kTilePad];
};

template <typename T, typename Acc>
struct alignas(16) TileSmem {
  TileBuf<T> buf[2];
  Acc rsum[kTileRows];
  Acc red[kTB / 32];
  unsigned long long bar[2];
  int flag;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: about 2^22 polls (each try_wait may itself suspend briefly)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

struct TileDesc {
  int r0, r1, k0, k1, mode;
};

__device__ __forceinline__ TileDesc load_tile(const int4 *__restrict__ tiles, int t) {
  int4 v = tiles[t];
  TileDesc d;
  d.r0 = v.x;
  d.r1 = v.y & kRowMask;
  d.mode = (int)((unsigned)v.y >> kModeShift);
  d.k0 = v.z;
  d.k1 = v.w;
  return d;
}

// aligned element range of [k0, k1) for 16-byte bulk copies of elements of `sz` bytes
__device__ __forceinline__ void aligned_range(int k0, int k1, int sz, int &a0, int &a1) {
  const int per = 16 / sz;
  a0 = k0 & ~(per - 1);
  a1 = (k1 + per - 1) & ~(per - 1);
}

// thread 0: start the copies of tile d into buffer b (caller guarantees the
// buffer is free and d is a staged tile with k1 > k0)
template <typename T, typename Acc>
__device__ __forceinline__ void issue_tile(TileSmem<T, Acc> &sm, int b, const TileDesc &d,
                                           const T *__restrict__ va, const int *__restrict__ ci) {
  int v0, v1, c0, c1;
  aligned_range(d.k0, d.k1, (int)sizeof(T), v0, v1);
  aligned_range(d.k0, d.k1, 4, c0, c1);
  const uint32_t bv = (uint32_t)(v1 - v0) * (uint32_t)sizeof(T);
  const uint32_t bc = (uint32_t)(c1 - c0) * 4u;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&sm.bar[b], bv + bc);
  bulk_copy_g2s(sm.buf[b].val, va + v0, bv, &sm.bar[b]);
  bulk_copy_g2s(sm.buf[b].ci, ci + c0, bc, &sm.bar[b]);
}

__device__ __forceinline__ bool staged(const TileDesc &d) {
  return d.mode != TM_LONG && d.k1 > d.k0;
}

template <typename Acc>
__device__ __forceinline__ Acc warp_allsum(Acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Walk the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; for each row r call
// epi.row(r, sum_k va[k] * vec[ci[k]]) once, with one thread per row.
// Returns false (after recording *err = code) if a bounded wait expired.
template <typename T, typename V, typename Acc, class Epi>
__device__ bool tile_spmv(TileSmem<T, Acc> &sm, const int4 *__restrict__ tiles, int ntiles,
                          const int *__restrict__ rp, const int *__restrict__ ci,
                          const T *__restrict__ va, const V *__restrict__ vec, Epi &epi,
                          int *err, int t_begin, int t_step) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
    sm.flag = 0;
  }
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};
  int pending = 0;  // bit q: a copy into buffer q is in flight (uniform)
  int b = 0;
  int t = t_begin;
  TileDesc cur;
  if (t < ntiles) {
    cur = load_tile(tiles, t);
    if (staged(cur)) {
      if (tid == 0) issue_tile(sm, b, cur, va, ci);
      pending |= 1 << b;
    }
  }
  bool ok = true;
  for (; t < ntiles; t += t_step) {
    const int tn = t + t_step;
    TileDesc nxt;
    if (tn < ntiles) {
      nxt = load_tile(tiles, tn);
      if (staged(nxt)) {
        if (tid == 0) issue_tile(sm, b ^ 1, nxt, va, ci);
        pending |= 1 << (b ^ 1);
      }
    }
    const int nrows = cur.r1 - cur.r0;
    if (cur.mode == TM_LONG) {
      // one long row straight from global memory, reduced by the whole CTA
      Acc s = 0;
      for (int k = cur.k0 + tid; k < cur.k1; k += kTB) s += (Acc)va[k] * (Acc)vec[ci[k]];
      s = warp_allsum(s);
      if (lane == 0) sm.red[warp] = s;
      __syncthreads();
      if (tid == 0) {
        Acc tot = 0;
        for (int w = 0; w < kTB / 32; ++w) tot += sm.red[w];
        sm.rsum[0] = tot;
      }
    } else {
      if (staged(cur)) {
        if (mbar_wait_bounded(&sm.bar[b], phase[b])) {
          phase[b] ^= 1u;
          pending &= ~(1 << b);
        } else {
          atomicOr(&sm.flag, 1);
        }
      }
      __syncthreads();
      if (sm.flag) {
        ok = false;
        break;
      }
      int v0, v1, c0, c1;
      aligned_range(cur.k0, cur.k1, (int)sizeof(T), v0, v1);
      aligned_range(cur.k0, cur.k1, 4, c0, c1);
      const T *sv = sm.buf[b].val - v0;  // index with global k
      const int *sc = sm.buf[b].ci - c0;
      if (cur.mode == TM_THREAD) {
        if (tid < nrows) {
          const int r = cur.r0 + tid;
          const int e = rp[r + 1];
          Acc s0 = 0, s1 = 0;
          int k = rp[r];
          for (; k + 1 < e; k += 2) {
            s0 += (Acc)sv[k] * (Acc)vec[sc[k]];
            s1 += (Acc)sv[k + 1] * (Acc)vec[sc[k + 1]];
          }
          if (k < e) s0 += (Acc)sv[k] * (Acc)vec[sc[k]];
          sm.rsum[tid] = s0 + s1;
        }
      } else if (cur.mode == TM_WARP) {
        for (int q = warp; q < nrows; q += kTB / 32) {
          const int r = cur.r0 + q;
          const int e = rp[r + 1];
          Acc s = 0;
          for (int k = rp[r] + lane; k < e; k += 32) s += (Acc)sv[k] * (Acc)vec[sc[k]];
          s = warp_allsum(s);
          if (lane == 0) sm.rsum[q] = s;
        }
      } else {  // TM_BLOCK: one row per tile, whole CTA
        Acc s = 0;
        for (int k = cur.k0 + tid; k < cur.k1; k += kTB) s += (Acc)sv[k] * (Acc)vec[sc[k]];
        s = warp_allsum(s);
        if (lane == 0) sm.red[warp] = s;
        __syncthreads();
        if (tid == 0) {
          Acc tot = 0;
          for (int w = 0; w < kTB / 32; ++w) tot += sm.red[w];
          sm.rsum[0] = tot;
        }
      }
    }
    __syncthreads();
    if (tid < nrows) epi.row(cur.r0 + tid, (double)sm.rsum[tid]);
    __syncthreads();  // buffer b and rsum are free again
    cur = nxt;
    b ^= 1;
  }
  if (!ok) {
    // record the failure, then let the copies this CTA started drain
    if (tid == 0) {
      atomicExch(err, 1);
      for (int q = 0; q < 2; ++q)
        if (pending & (1 << q)) mbar_wait_bounded(&sm.bar[q], phase[q]);
    }
    __syncthreads();
  }
  return ok;
}

}  // namespace gb300lp
