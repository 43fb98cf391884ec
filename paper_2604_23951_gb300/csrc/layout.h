// Device layout of one LP, built on the host: rows of A and of A^T sorted by
// length (longest first) and renumbered, the stored transpose, and the warp
// tile tables of spmv_warp.cuh.  Shared by the single-LP upload and the
// batch server's request packing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
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

struct Layout {
  int m = 0, n = 0;
  long long nnz = 0;
  std::vector<int> rperm, cperm;  // new -> old
  std::vector<int> arp, aci, trp, tci;  // CSR of the permuted A and A^T (padded)
  std::vector<double> av, tv;
  std::vector<int2> tA, tT;  // warp tiles
  int nlongA = 0, nlongT = 0;
  std::vector<double> c0, lx0, ux0, lc0, uc0;  // permuted problem vectors
  std::vector<double> pv0;  // power-iteration fallback start (power_start of cperm)
  double bnorm = 0, cnorm = 0, off = 0;
};

void build_layout(const HostLP &h, Layout &L);

// the row order and warp tiles of one matrix (exposed for the layout checks)
void plan_tiles(const std::vector<int64_t> &len, std::vector<int> &perm,
                std::vector<int2> &tiles, int &nlong);

}  // namespace gb300lp
