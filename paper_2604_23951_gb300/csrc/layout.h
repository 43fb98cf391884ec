// Device layout of one LP, built on the host: rows of A and of A^T sorted by
// length (longest first) and renumbered, the stored transpose, and the warp
// tile tables of spmv_warp.cuh.  Shared by the single-LP upload and the
// batch server's request packing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <utility>
#include <vector>

#include "lp_internal.h"

namespace gb300lp {

constexpr int kTilePad = 8;  // value / index arrays padded past nnz

#if defined(__CUDACC__)
#define GB300LP_HD __host__ __device__
#else
#define GB300LP_HD
#endif

// Fallback start vector of the power iteration for ||A||_2 (which starts
// from all-ones / sqrt(n) and continues from this vector when a step gives
// zero: all-ones is orthogonal to A's row space when the rows of A sum to
// zero, e.g. A = [1, -1]).  Entry of original column j:
// (0.5 + h(j) / 2^32) / sqrt(n) with the multiplicative hash
// h(j) = j * 2654435761 mod 2^32.  Indexed by the ORIGINAL column, so every
// storage order uses the same vector.
GB300LP_HD inline double power_start(int j, double inv_sqrt_n) {
  const unsigned h = (unsigned)j * 2654435761u;
  return (0.5 + (double)h * (1.0 / 4294967296.0)) * inv_sqrt_n;
}

// Shape of the warp tiles over one matrix's length-sorted rows (runtime
// parameters of the row plan; the autotuner searches them).
//   run_max   most entries one lane owns in a row: a tile whose longest row
//             has L entries gives each row 2^v lanes, v the least with
//             2^v * run_max >= L (at most 32 lanes);
//   tile_nnz  nonzeros a tile aims at: L <= tile_nnz / 32 gives 32 rows,
//             longer rows tile_nnz / L rows (at least 1);
//   segmented rows longer than 32 * run_max are cut into segments of
//             32 * run_max entries, one warp each, whose partial sums the
//             last warp to finish a row adds up (single-LP path); otherwise
//             (batch path) rows up to kCtaRow get a single-row tile and longer
//             rows are reduced by a whole CTA (nlong of them, first).
// A vector whose new elements are left uninitialised (the large arrays of a
// layout are written in full right after they are sized).
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U> &) {}
  template <class U>
  void construct(U *p) noexcept {
    ::new (static_cast<void *>(p)) U;
  }
  template <class U, class... A>
  void construct(U *p, A &&...a) {
    ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using UninitVec = std::vector<T, UninitAlloc<T>>;

struct TileShape {
  int run_max = 8;
  int tile_nnz = 512;
  bool segmented = false;
};

// the tile table of one matrix under one shape
struct TilePlan {
  std::vector<int2> tiles;
  int nlong = 0;                // CTA rows (unsegmented shapes)
  int nsegrows = 0;             // segmented rows (the first nsegrows rows)
  std::vector<int> seg_base;    // nsegrows + 1: row r's segments are
                                // seg_base[r] .. seg_base[r + 1] - 1
  int seg_len = 0;              // entries per segment
};

struct Layout {
  int m = 0, n = 0;
  long long nnz = 0;
  std::vector<int> rperm, cperm;  // new -> old
  std::vector<int> arp, trp;            // row offsets of the permuted A and A^T
  UninitVec<int> aci, tci;              // their indices and values (padded past
  UninitVec<double> av, tv;             // nnz with zeros)
  TilePlan pA, pT;  // tiles under the shape build_layout was given
  std::vector<double> c0, lx0, ux0, lc0, uc0;  // permuted problem vectors
  std::vector<double> pv0;  // power-iteration fallback start (power_start of cperm)
  double bnorm = 0, cnorm = 0, off = 0;
};

// Rows are renumbered longest first (stable), whatever the shape, so one
// stored matrix serves every tile shape.
void build_layout(const HostLP &h, Layout &L, const TileShape &shape);

// the length order of a matrix's rows (perm[new] = old)
void sort_rows(const std::vector<int64_t> &len, std::vector<int> &perm);

// the tile table of rows already in that order (sorted[r] = length of row r)
void plan_tiles(const std::vector<int64_t> &sorted, const TileShape &shape, TilePlan &plan);

}  // namespace gb300lp
