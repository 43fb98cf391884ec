// Host construction of the device layout (see layout.h).
#include "layout.h"

#include <algorithm>
#include <cmath>
#include <string>

#include "spmv_warp.cuh"

namespace gb300lp {

// Order rows for the warp engine (stable within a class): rows longer than
// kCtaRow first (nlong of them, one whole CTA each), then rows longer than
// kLongRow (a single-row warp tile each), then the rest by length, longest
// first, cut into warp tiles of at most 32 rows and about kWarpTileNnz
// nonzeros.  A tile's lanes per row 2^v is the least with 2^v * kWarpItems
// >= its longest row L, and its entries per lane nit = ceil(L / 2^v).
void plan_tiles(const std::vector<int64_t> &len, std::vector<int> &perm,
                std::vector<int2> &tiles, int &nlong) {
  const int rows = (int)len.size();
  // key: the length for rows up to kLongRow, kLongRow + 1 for warp-long
  // rows, kLongRow + 2 for CTA rows; counting sort by descending key
  auto key = [](int64_t L) -> int {
    if (L > kCtaRow) return kLongRow + 2;
    if (L > kLongRow) return kLongRow + 1;
    return (int)L;
  };
  const int nkeys = kLongRow + 3;
  std::vector<int> cnt(nkeys, 0);
  for (int64_t L : len) cnt[key(L)]++;
  std::vector<int> start(nkeys, 0);
  int acc = 0;
  for (int k = nkeys - 1; k >= 0; --k) {
    start[k] = acc;
    acc += cnt[k];
  }
  perm.assign(rows, 0);
  for (int r = 0; r < rows; ++r) perm[start[key(len[r])]++] = r;
  tiles.clear();
  int i = 0;
  while (i < rows && len[perm[i]] > kCtaRow) ++i;
  nlong = i;
  while (i < rows && len[perm[i]] > kLongRow) {
    tiles.push_back(pack_wtile(i, 1, 5, kWarpItems));
    ++i;
  }
  while (i < rows) {
    const int64_t L = len[perm[i]];
#ifndef GB300_MIN_VLOG
#define GB300_MIN_VLOG 0
#endif
    int vlog = GB300_MIN_VLOG;
    while ((int64_t(1) << vlog) * kWarpItems < L) ++vlog;
    const int vl = 1 << vlog;
    const int nit = (int)std::max<int64_t>(1, (L + vl - 1) / vl);
    int nr = (int)std::max<int64_t>(
        1, std::min<int64_t>(32, kWarpTileNnz / std::max<int64_t>(L, 1)));
    nr = std::min(nr, rows - i);
    tiles.push_back(pack_wtile(i, nr, vlog, nit));
    i += nr;
  }
}

void build_layout(const HostLP &h, Layout &L) {
  const int m = h.m, n = h.n;
  const long long nnz = h.nnz();
  L.m = m;
  L.n = n;
  L.nnz = nnz;
  std::vector<int64_t> rlen(m), clen(n, 0);
  for (int i = 0; i < m; ++i) rlen[i] = h.row_ptr[i + 1] - h.row_ptr[i];
  for (long long k = 0; k < nnz; ++k) clen[h.col_idx[k]]++;
  plan_tiles(rlen, L.rperm, L.tA, L.nlongA);
  plan_tiles(clen, L.cperm, L.tT, L.nlongT);
  std::vector<int> cinv(n);
  for (int j = 0; j < n; ++j) cinv[L.cperm[j]] = j;
  L.arp.assign(m + 1, 0);
  L.aci.assign(nnz + kTilePad, 0);
  L.av.assign(nnz + kTilePad, 0.0);
  for (int i = 0; i < m; ++i) {
    int o = L.rperm[i];
    L.arp[i + 1] = L.arp[i] + (int)rlen[o];
    int w = L.arp[i];
    for (int64_t k = h.row_ptr[o]; k < h.row_ptr[o + 1]; ++k, ++w) {
      L.aci[w] = cinv[h.col_idx[k]];
      L.av[w] = h.val[k];
    }
  }
  // transpose of the permuted A: rows in new column order, entries by new row
  L.trp.assign(n + 1, 0);
  L.tci.assign(nnz + kTilePad, 0);
  L.tv.assign(nnz + kTilePad, 0.0);
  for (int j = 0; j < n; ++j) L.trp[j + 1] = L.trp[j] + (int)clen[L.cperm[j]];
  {
    std::vector<int> cur(L.trp.begin(), L.trp.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int k = L.arp[i]; k < L.arp[i + 1]; ++k) {
        int j = L.aci[k];
        L.tci[cur[j]] = i;
        L.tv[cur[j]] = L.av[k];
        ++cur[j];
      }
  }
  L.c0.resize(n);
  L.lx0.resize(n);
  L.ux0.resize(n);
  L.pv0.resize(n);
  L.lc0.resize(m);
  L.uc0.resize(m);
  const double inv_sqrt_n = n > 0 ? 1.0 / std::sqrt((double)n) : 0.0;
  for (int j = 0; j < n; ++j) {
    int o = L.cperm[j];
    L.c0[j] = h.c[o];
    L.lx0[j] = h.col_lo[o];
    L.ux0[j] = h.col_hi[o];
    L.pv0[j] = power_start(o, inv_sqrt_n);
  }
  for (int i = 0; i < m; ++i) {
    int o = L.rperm[i];
    L.lc0[i] = h.row_lo[o];
    L.uc0[i] = h.row_hi[o];
  }
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

extern "C" int lp_plan_rows(int32_t rows, const int64_t *len, int32_t *perm, int32_t *tiles,
                            int32_t tile_cap, int32_t *ntiles, int32_t *nlong) {
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
  std::vector<int2> t;
  int nl = 0;
  plan_tiles(L, p, t, nl);
  *ntiles = (int32_t)t.size();
  *nlong = nl;
  if ((int64_t)t.size() > tile_cap) {
    set_last_error("lp_plan_rows: tile_cap too small");
    return LP_ERR_INVALID;
  }
  std::copy(p.begin(), p.end(), perm);
  for (size_t k = 0; k < t.size(); ++k) {
    tiles[2 * k] = t[k].x;
    tiles[2 * k + 1] = t[k].y;
  }
  return LP_OK;
}
