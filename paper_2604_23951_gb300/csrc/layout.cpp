// Host construction of the device layout (see layout.h).
#include "layout.h"

#include <algorithm>
#include <cmath>

#include "spmv_warp.cuh"

namespace gb300lp {

// Sort rows by length (longest first, stable).  Rows longer than kLongRow
// come first (nlong of them, one whole-CTA reduction each); the rest are cut
// into warp tiles of at most 32 rows and about kWarpTileNnz nonzeros, each
// reducing its rows with 2^v lanes so no lane owns more than kWarpItems.
static void plan_tiles(const std::vector<int64_t> &len, std::vector<int> &perm,
                       std::vector<int2> &tiles, int &nlong) {
  const int rows = (int)len.size();
  int64_t lmax = 0;
  for (int64_t L : len) lmax = std::max(lmax, L);
  const int64_t cap = std::min<int64_t>(lmax, (int64_t)kLongRow + 1);
  std::vector<int> cnt(cap + 2, 0);
  for (int64_t L : len) cnt[std::min(L, cap)]++;
  std::vector<int> start(cap + 2, 0);
  int acc = 0;
  for (int64_t L = cap; L >= 0; --L) {
    start[L] = acc;
    acc += cnt[L];
  }
  perm.assign(rows, 0);
  for (int r = 0; r < rows; ++r) perm[start[std::min(len[r], cap)]++] = r;
  tiles.clear();
  int i = 0;
  while (i < rows && len[perm[i]] > kLongRow) ++i;
  nlong = i;
  while (i < rows) {
    const int64_t L = len[perm[i]];
    int vlog = 0;
    const int64_t per = (L + kWarpItems - 1) / kWarpItems;
    while ((1LL << vlog) < per && vlog < 5) ++vlog;
    int nr = (int)std::max<int64_t>(
        1, std::min<int64_t>(32, kWarpTileNnz / std::max<int64_t>(L, 1)));
    nr = std::min(nr, rows - i);
    tiles.push_back(make_int2(i, nr | (vlog << 8)));
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
  L.lc0.resize(m);
  L.uc0.resize(m);
  for (int j = 0; j < n; ++j) {
    int o = L.cperm[j];
    L.c0[j] = h.c[o];
    L.lx0[j] = h.col_lo[o];
    L.ux0[j] = h.col_hi[o];
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
