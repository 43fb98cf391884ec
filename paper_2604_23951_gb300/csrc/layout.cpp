// Host construction of the device layout (see layout.h).
#include "layout.h"

#include "host_parallel.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "spmv_warp.cuh"

namespace gb300lp {

// Rows longest first, stable (counting sort on the length when the longest
// row allows it, a stable comparison sort otherwise).
void sort_rows(const std::vector<int64_t> &len, std::vector<int> &perm) {
  const int rows = (int)len.size();
  perm.assign(rows, 0);
  int64_t lmax = 0;
  for (int64_t L : len) lmax = std::max(lmax, L);
  if (lmax <= (int64_t(1) << 22)) {
    std::vector<int> cnt(lmax + 2, 0);
    for (int64_t L : len) cnt[L]++;
    // start of each length, longest first
    std::vector<int> start(lmax + 2, 0);
    int acc = 0;
    for (int64_t L = lmax; L >= 0; --L) {
      start[L] = acc;
      acc += cnt[L];
    }
    for (int r = 0; r < rows; ++r) perm[start[len[r]]++] = r;
  } else {
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(),
                     [&](int a, int b) { return len[a] > len[b]; });
  }
}

// Tiles over rows in length order (sorted[r] = length of row r).  Rows
// longer than 32 * run_max come first: segmented (one tile per segment,
// {row, INT_MIN | segment index}) or, unsegmented, rows longer than kCtaRow
// as CTA rows and the others as single-row tiles.  The rest is cut into
// tiles of up to 32 rows and about tile_nnz nonzeros (a tile whose first
// row is longer than 8 ends before a row of less than half its length); in
// a tile whose longest row has L entries each row gets 2^v lanes (least v with 2^v * run_max >= L)
// and a lane walks its share in c = ceil(L / (2^v * 8)) chunks of
// nit = ceil(L / (2^v * c)) <= 8 entries (balanced chunks: no lane pads more
// than one chunk step).
void plan_tiles(const std::vector<int64_t> &sorted, const TileShape &shape, TilePlan &plan) {
  const int rows = (int)sorted.size();
  const int rmax = std::max(1, std::min(shape.run_max, 64));
  const int64_t llong = 32LL * rmax;
  plan.tiles.clear();
  plan.seg_base.assign(1, 0);
  plan.nlong = 0;
  plan.nsegrows = 0;
  plan.seg_len = 0;
  int i = 0;
  if (shape.segmented) {
    plan.seg_len = (int)llong;
    int g = 0;
    while (i < rows && sorted[i] > llong) {
      const int nseg = (int)((sorted[i] + llong - 1) / llong);
      for (int s = 0; s < nseg; ++s)
        plan.tiles.push_back(make_int2(i, (int)(0x80000000u | (unsigned)(g + s))));
      g += nseg;
      plan.seg_base.push_back(g);
      ++i;
    }
    plan.nsegrows = i;
  } else {
    while (i < rows && sorted[i] > kCtaRow) ++i;
    plan.nlong = i;
    while (i < rows && sorted[i] > llong) {
      const int nit = (int)std::min<int64_t>(kWarpItems, (sorted[i] + 31) / 32);
      plan.tiles.push_back(pack_wtile(i, 1, 5, std::max(1, nit)));
      ++i;
    }
  }
  const int64_t tnnz = std::max(32, shape.tile_nnz);
  while (i < rows) {
    const int64_t L = sorted[i];
    int vlog = 0;
    while ((int64_t(1) << vlog) * rmax < L && vlog < 5) ++vlog;
    const int64_t vl = int64_t(1) << vlog;
    const int64_t chunks = std::max<int64_t>(1, (L + vl * kWarpItems - 1) / (vl * kWarpItems));
    const int nit = (int)std::max<int64_t>(1, (L + vl * chunks - 1) / (vl * chunks));
    int nr = (int)std::max<int64_t>(1, std::min<int64_t>(32, tnnz / std::max<int64_t>(L, 1)));
    nr = std::min(nr, rows - i);
    // rows much shorter than the first would idle most of their lanes
    for (int k = 1; k < nr; ++k)
      if (L > kWarpItems && 2 * sorted[i + k] < L) {
        nr = k;
        break;
      }
    plan.tiles.push_back(pack_wtile(i, nr, vlog, nit));
    i += nr;
  }
}

void build_layout(const HostLP &h, Layout &L, const TileShape &shape) {
  const int m = h.m, n = h.n;
  const long long nnz = h.nnz();
  L.m = m;
  L.n = n;
  L.nnz = nnz;
  // the O(nnz) passes run on host threads for large matrices; every pass
  // gives the same result as in one thread (chunks own disjoint outputs)
  const bool par = nnz >= 1000000;
  std::vector<int64_t> rlen(m), clen(n, 0);
  for (int i = 0; i < m; ++i) rlen[i] = h.row_ptr[i + 1] - h.row_ptr[i];
  // column counts: a chunk of columns counts its own entries in one scan
  host_parallel_chunks((size_t)n, par, [&](unsigned, size_t j0, size_t j1) {
    const int32_t lo = (int32_t)j0, hi = (int32_t)j1;
    for (long long k = 0; k < nnz; ++k) {
      const int32_t j = h.col_idx[k];
      if (j >= lo && j < hi) clen[j]++;
    }
  });
  sort_rows(rlen, L.rperm);
  sort_rows(clen, L.cperm);
  {
    std::vector<int64_t> sr(m), sc(n);
    for (int i = 0; i < m; ++i) sr[i] = rlen[L.rperm[i]];
    for (int j = 0; j < n; ++j) sc[j] = clen[L.cperm[j]];
    plan_tiles(sr, shape, L.pA);
    plan_tiles(sc, shape, L.pT);
  }
  std::vector<int> cinv(n);
  for (int j = 0; j < n; ++j) cinv[L.cperm[j]] = j;
  L.arp.assign(m + 1, 0);
  L.aci.resize(nnz + kTilePad);
  L.av.resize(nnz + kTilePad);
  for (int q = 0; q < kTilePad; ++q) {
    L.aci[nnz + q] = 0;
    L.av[nnz + q] = 0.0;
  }
  for (int i = 0; i < m; ++i) L.arp[i + 1] = L.arp[i] + (int)rlen[L.rperm[i]];
  host_parallel_chunks((size_t)m, par, [&](unsigned, size_t i0, size_t i1) {
    for (size_t i = i0; i < i1; ++i) {
      const int o = L.rperm[i];
      int w = L.arp[i];
      for (int64_t k = h.row_ptr[o]; k < h.row_ptr[o + 1]; ++k, ++w) {
        L.aci[w] = cinv[h.col_idx[k]];
        L.av[w] = h.val[k];
      }
    }
  });
  // transpose of the permuted A: rows in new column order, entries by new
  // row; a chunk of new columns scans the rows in order and places its own
  // entries
  L.trp.assign(n + 1, 0);
  L.tci.resize(nnz + kTilePad);
  L.tv.resize(nnz + kTilePad);
  for (int q = 0; q < kTilePad; ++q) {
    L.tci[nnz + q] = 0;
    L.tv[nnz + q] = 0.0;
  }
  for (int j = 0; j < n; ++j) L.trp[j + 1] = L.trp[j] + (int)clen[L.cperm[j]];
  {
    std::vector<int> cur(L.trp.begin(), L.trp.end() - 1);
    host_parallel_chunks((size_t)n, par, [&](unsigned, size_t j0, size_t j1) {
      const int lo = (int)j0, hi = (int)j1;
      for (int i = 0; i < m; ++i)
        for (int k = L.arp[i]; k < L.arp[i + 1]; ++k) {
          const int j = L.aci[k];
          if (j < lo || j >= hi) continue;
          L.tci[cur[j]] = i;
          L.tv[cur[j]] = L.av[k];
          ++cur[j];
        }
    });
  }
  L.c0.resize(n);
  L.lx0.resize(n);
  L.ux0.resize(n);
  L.pv0.resize(n);
  L.lc0.resize(m);
  L.uc0.resize(m);
  const double inv_sqrt_n = n > 0 ? 1.0 / std::sqrt((double)n) : 0.0;
  host_parallel_chunks((size_t)n, par, [&](unsigned, size_t j0, size_t j1) {
    for (size_t j = j0; j < j1; ++j) {
      const int o = L.cperm[j];
      L.c0[j] = h.c[o];
      L.lx0[j] = h.col_lo[o];
      L.ux0[j] = h.col_hi[o];
      L.pv0[j] = power_start(o, inv_sqrt_n);
    }
  });
  host_parallel_chunks((size_t)m, par, [&](unsigned, size_t i0, size_t i1) {
    for (size_t i = i0; i < i1; ++i) {
      const int o = L.rperm[i];
      L.lc0[i] = h.row_lo[o];
      L.uc0[i] = h.row_hi[o];
    }
  });
  // norms of the unscaled data for the relative KKT error
  double bn2 = 0, cn2 = 0;
  for (int i = 0; i < m; ++i) {
    bool lf = std::isfinite(L.lc0[i]), uf = std::isfinite(L.uc0[i]);
    if (lf) bn2 += L.lc0[i] * L.lc0[i];
    if (uf && !(lf && L.lc0[i] == L.uc0[i])) bn2 += L.uc0[i] * L.uc0[i];
  }
  for (int j = 0; j < n; ++j) cn2 += L.c0[j] * L.c0[j];
  L.bnorm = std::sqrt(bn2);
  L.cnorm = std::sqrt(cn2);
  L.off = h.off;
}

}  // namespace gb300lp

namespace gb300lp {
void set_last_error(const std::string &m);
}

// the row plan of one matrix under a shape (shared by the two C entry points)
static int plan_rows_common(int32_t rows, const int64_t *len, const gb300lp::TileShape &shape,
                            int32_t *perm, int32_t *tiles, int32_t tile_cap, int32_t *ntiles,
                            int32_t *nlong, int32_t *seg_base, int32_t seg_cap,
                            int32_t *nsegrows) {
  using namespace gb300lp;
  if (rows < 0 || (rows > 0 && (!len || !perm)) || !ntiles || !nlong || tile_cap < 0 ||
      (tile_cap > 0 && !tiles)) {
    set_last_error("lp_plan_rows: invalid argument");
    return LP_ERR_INVALID;
  }
  std::vector<int64_t> L(len, len + rows);
  for (int64_t v : L)
    if (v < 0) {
      set_last_error("lp_plan_rows: negative row length");
      return LP_ERR_INVALID;
    }
  std::vector<int> p;
  sort_rows(L, p);
  std::vector<int64_t> sl(rows);
  for (int r = 0; r < rows; ++r) sl[r] = L[p[r]];
  TilePlan plan;
  plan_tiles(sl, shape, plan);
  *ntiles = (int32_t)plan.tiles.size();
  *nlong = plan.nlong;
  if (nsegrows) *nsegrows = plan.nsegrows;
  if ((int64_t)plan.tiles.size() > tile_cap) {
    set_last_error("lp_plan_rows: tile_cap too small");
    return LP_ERR_INVALID;
  }
  if (seg_base) {
    if ((int64_t)plan.seg_base.size() > seg_cap) {
      set_last_error("lp_plan_rows: seg_cap too small");
      return LP_ERR_INVALID;
    }
    std::copy(plan.seg_base.begin(), plan.seg_base.end(), seg_base);
  }
  std::copy(p.begin(), p.end(), perm);
  for (size_t k = 0; k < plan.tiles.size(); ++k) {
    tiles[2 * k] = plan.tiles[k].x;
    tiles[2 * k + 1] = plan.tiles[k].y;
  }
  return LP_OK;
}

extern "C" int lp_plan_rows(int32_t rows, const int64_t *len, int32_t *perm, int32_t *tiles,
                            int32_t tile_cap, int32_t *ntiles, int32_t *nlong) {
  gb300lp::TileShape shape;  // the batch path's shape: run_max 8, 512 nonzeros, CTA rows
  return plan_rows_common(rows, len, shape, perm, tiles, tile_cap, ntiles, nlong, nullptr, 0,
                          nullptr);
}

extern "C" int lp_plan_rows_shape(int32_t rows, const int64_t *len, int32_t run_max,
                                  int32_t tile_nnz, int32_t segmented, int32_t *perm,
                                  int32_t *tiles, int32_t tile_cap, int32_t *ntiles,
                                  int32_t *nlong, int32_t *seg_base, int32_t seg_cap,
                                  int32_t *nsegrows) {
  if (run_max < 1 || run_max > 64 || tile_nnz < 32) {
    gb300lp::set_last_error("lp_plan_rows_shape: run_max must be 1..64, tile_nnz >= 32");
    return LP_ERR_INVALID;
  }
  gb300lp::TileShape shape;
  shape.run_max = run_max;
  shape.tile_nnz = tile_nnz;
  shape.segmented = segmented != 0;
  return plan_rows_common(rows, len, shape, perm, tiles, tile_cap, ntiles, nlong, seg_base,
                          seg_cap, nsegrows);
}
