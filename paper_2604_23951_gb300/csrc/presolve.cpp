// Host presolve / postsolve for eq. (1): the simple ("fast") explorers of
// Table 1 applied through the reductions of Sec. 2.1, in rounds (Sec. 3.2),
// with A stored both row-wise and column-wise with per-row / per-column
// slack for fill-in (Sec. 3.2).
//
// Rules, schedule and postsolve formulas:
//   round = empty rows -> empty cols -> fixed cols -> singleton rows ->
//           redundant rows / dominated sides -> doubleton equalities ->
//           column singletons in inequality rows (made equalities) ->
//           free (or implied-free) column singletons in equality rows ->
//           variable locks (weak dual fixing, Sec. 2.3);
//   each pass scans candidates in increasing index order; round 1 scans
//   everything, later rounds what the previous round dirtied.  A round in
//   which these fast passes change nothing runs the medium explorer
//   parallel rows over every row; stop when that finds nothing either, or
//   after max_rounds.
//   Infeasibility when a lower bound exceeds an upper one by more than 1e-9;
//   coefficients below 1e-12 in magnitude after an update are dropped; the
//   rules that read a cost's sign (empty columns, variable locks, column
//   singletons in inequality rows) take |c_j| <= 1e-12 * max(1, max |c| of
//   the input) as zero, since substitutions leave rounding residue in c;
//   activities sum a row's entries in increasing column order, compared with
//   the row bounds exactly.  Arithmetic is plain IEEE double (the library is
//   built with -ffp-contract=off), so the decisions are reproducible.
//
// Postsolve keeps c - A^T y - z = 0 (second line of eq. (2)) for every
// intermediate problem:
//   empty / redundant row:   y_i = 0
//   dropped row side:        nothing
//   fixed / empty column v:  x_j = v, z_j = c_j - sum_i a_ij y_i   (Sec. 2.1)
//   singleton row a x_j:     y_i = z_j / a, z_j = 0 when z_j's sign points at
//                            a bound that came from the row, else y_i = 0
//   doubleton a_j x_j + a_k x_k = b:  x_j = (b - a_k x_k) / a_j;
//                            D_j = c_j - sum_{r != i} a_rj y_r;
//                            bound of x_k active and transferred from x_j:
//                              y_i = (z_k + (a_k / a_j) D_j) / a_k,
//                              z_j = D_j - a_j y_i, z_k = 0;
//                            otherwise y_i = D_j / a_j, z_j = 0
//   free column singleton:   x_j = (b - sum_{r != j} a_ir x_r) / a_ij,
//                            y_i = c_j / a_ij, z_j = 0
//   inequality row i made an equality at one side:  a y_i of the other sign
//                            is set to 0 and z_r -= a_ir * (0 - y_i) over the
//                            row's entries at that time
//   bound of x_j tightened from row i:  z_j of the sign that points at the
//                            tightened bound moves to the row: y_i += z_j /
//                            a_ij, z_r -= a_ir z_j / a_ij over its entries
//   parallel column k (a_k = s a_j, c_k = s c_j) merged into x_j + s x_k = v:
//                            x_k = proj_[l_k,u_k](0), x_j = v - s x_k; if x_j
//                            leaves its bounds it takes the violated one and
//                            x_k = proj((v - x_j) / s); z_k = s z_j
//   parallel row k (a_k = s a_i) merged into row i:  y_k = y_i / s, y_i = 0
//                            when y_i's sign points at a side that came
//                            strictly from row k; else y_k = 0
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <limits>
#include <thread>
#include <vector>

#include "lp_internal.h"

namespace gb300lp {
namespace {

constexpr double kFeasTol = 1e-9;
constexpr double kDropTol = 1e-12;
constexpr double kCostTol = 1e-12;
constexpr double kInf = std::numeric_limits<double>::infinity();

enum RecKind {
  REC_EMPTY_ROW = 0,
  REC_REDUNDANT_ROW = 1,
  REC_DROP_SIDE = 2,
  REC_FIX_COL = 3,
  REC_SINGLETON_ROW = 4,
  REC_DOUBLETON = 5,
  REC_FREE_COL = 6,
  REC_ROW_TO_EQ = 7,
  REC_PARALLEL_ROW = 8,
  REC_TIGHTEN = 9,
  REC_PARALLEL_COL = 10,
};

enum CountIdx {
  C_EMPTY_ROW = 0, C_EMPTY_COL, C_FIXED_COL, C_SINGLETON_ROW, C_REDUNDANT_ROW,
  C_DROPPED_SIDE, C_DOUBLETON, C_FREE_COL, C_DUAL_FIX, C_INEQ_TO_EQ, C_PARALLEL_ROW,
  C_TIGHTENED, C_PARALLEL_COL, C_DUAL_PROP,
};

constexpr double kDualPropTol = 1e-9;  // a dual / reduced cost this far from 0 has a sign

// Primal propagation: an implied bound replaces a finite one when tighter by
// more than kPropStep * max(1, |bound|), an infinite one when its magnitude
// is at most kPropMaxBound.
constexpr double kPropStep = 1e-3;
constexpr double kPropMaxBound = 1e6;
constexpr int kPropSweeps = 2;  // propagation sweeps per presolve

// Parallel rows: coefficients agree to this relative tolerance, and a row is
// compared with at most this many earlier unmerged rows of its column pattern.
constexpr double kParTol = 1e-12;
constexpr int kParCandidates = 32;

// Worker threads that are always joined, also when an exception unwinds the
// caller; work whose thread cannot be started runs on the calling thread.
class ThreadGroup {
 public:
  template <class F>
  void run(const F &f, size_t a, size_t b) {
    try {
      ts_.emplace_back(f, a, b);
    } catch (const std::exception &) {
      f(a, b);
    }
  }
  void join() {
    for (std::thread &t : ts_)
      if (t.joinable()) t.join();
  }
  ~ThreadGroup() { join(); }

 private:
  std::vector<std::thread> ts_;
};

// Sorted sparse vectors in one pool, each with spare capacity.  A vector that
// outgrows its capacity moves to the end of the pool with twice the room.
struct SlackStore {
  std::vector<int64_t> start;
  std::vector<int32_t> len, cap;
  std::vector<int32_t> idx;
  std::vector<double> val;

  void init(int32_t count, const std::vector<int32_t> &lens) {
    start.assign(count, 0);
    len.assign(count, 0);
    cap.assign(count, 0);
    int64_t total = 0;
    for (int32_t r = 0; r < count; ++r) {
      start[r] = total;
      cap[r] = lens[r] + 2 + lens[r] / 4;
      total += cap[r];
    }
    // room for vectors that outgrow their slack to move to the end without
    // reallocating (and copying) the whole pool; reserved pages cost nothing
    // until they are used
    idx.reserve(total + total / 4 + 4096);
    val.reserve(total + total / 4 + 4096);
    idx.assign(total, 0);
    val.assign(total, 0.0);
  }
  // position of key in vector r, or -(insertion point) - 1
  int32_t find(int32_t r, int32_t key) const {
    const int32_t *p = idx.data() + start[r];
    int32_t lo = 0, hi = len[r];
    while (lo < hi) {
      int32_t mid = (lo + hi) >> 1;
      if (p[mid] < key) lo = mid + 1; else hi = mid;
    }
    if (lo < len[r] && p[lo] == key) return lo;
    return -lo - 1;
  }
  void erase_at(int32_t r, int32_t pos) {
    const int64_t s = start[r];
    const int32_t tail = len[r] - pos - 1;
    if (tail > 0) {
      std::memmove(&idx[s + pos], &idx[s + pos + 1], sizeof(int32_t) * tail);
      std::memmove(&val[s + pos], &val[s + pos + 1], sizeof(double) * tail);
    }
    --len[r];
  }
  void erase(int32_t r, int32_t key) {
    int32_t p = find(r, key);
    if (p >= 0) erase_at(r, p);
  }
  void grow(int32_t r) {
    int32_t ncap = std::max(4, cap[r] * 2);
    int64_t ns = (int64_t)idx.size();
    idx.resize(ns + ncap);
    val.resize(ns + ncap);
    for (int32_t q = 0; q < len[r]; ++q) {
      idx[ns + q] = idx[start[r] + q];
      val[ns + q] = val[start[r] + q];
    }
    start[r] = ns;
    cap[r] = ncap;
  }
  // insert or overwrite
  void put(int32_t r, int32_t key, double v) {
    int32_t p = find(r, key);
    if (p >= 0) {
      val[start[r] + p] = v;
      return;
    }
    int32_t ins = -p - 1;
    if (len[r] == cap[r]) grow(r);
    const int64_t s = start[r];
    const int32_t tail = len[r] - ins;
    if (tail > 0) {
      std::memmove(&idx[s + ins + 1], &idx[s + ins], sizeof(int32_t) * tail);
      std::memmove(&val[s + ins + 1], &val[s + ins], sizeof(double) * tail);
    }
    idx[s + ins] = key;
    val[s + ins] = v;
    ++len[r];
  }
  double get(int32_t r, int32_t key, double dflt) const {
    int32_t p = find(r, key);
    return p >= 0 ? val[start[r] + p] : dflt;
  }
};

struct Presolver {
  int32_t m, n;
  SlackStore rows, cols;
  std::vector<double> c, lo, hi, lx, ux;
  double off;
  double cost_tol = kCostTol;
  std::vector<uint8_t> row_on, col_on;
  std::vector<uint8_t> dmark_r, dmark_c;
  std::vector<uint8_t> fixmark, rmark;  // scratch of the batched fixed-column pass
  std::vector<double> prop_lo, prop_hi;   // scratch of primal propagation (one row)
  std::vector<int32_t> dlist_r, dlist_c;
  bool changed = false;
  int32_t status = LP_PRESOLVE_REDUCED;
  PresolveOutcome *po;

  explicit Presolver(const HostLP &in, PresolveOutcome *out) : po(out) {
    m = in.m;
    n = in.n;
    std::vector<int32_t> rl(m), cl(n, 0);
    for (int32_t i = 0; i < m; ++i) {
      int32_t cnt = 0;
      for (int64_t k = in.row_ptr[i]; k < in.row_ptr[i + 1]; ++k)
        if (in.val[k] != 0.0) { ++cnt; ++cl[in.col_idx[k]]; }
      rl[i] = cnt;
    }
    // Input rows are sorted by column and rows arrive in order, so both
    // stores fill by appends.  The column store is a scatter: it is built
    // by several threads, each owning a contiguous range of columns and
    // scanning all rows for the entries of its range (every column still
    // receives its entries in row order), while this thread fills the rows.
    cols.init(n, cl);
    const int64_t nnz_in = in.row_ptr.empty() ? 0 : in.row_ptr.back();
    const unsigned ncb =
        nnz_in >= 1000000 ? std::min(8u, std::max(1u, std::thread::hardware_concurrency())) : 1u;
    auto fill_cols = [&](size_t j0, size_t j1) {
      for (int32_t i = 0; i < m; ++i)
        for (int64_t k = in.row_ptr[i]; k < in.row_ptr[i + 1]; ++k) {
          const int32_t j = in.col_idx[k];
          if ((size_t)j < j0 || (size_t)j >= j1) continue;
          const double v = in.val[k];
          if (v == 0.0) continue;
          cols.idx[cols.start[j] + cols.len[j]] = i;
          cols.val[cols.start[j] + cols.len[j]] = v;
          ++cols.len[j];
        }
    };
    ThreadGroup col_builders;
    for (unsigned t = 0; t < ncb; ++t)
      col_builders.run(fill_cols, (size_t)n * t / ncb, (size_t)n * (t + 1) / ncb);
    rows.init(m, rl);
    for (int32_t i = 0; i < m; ++i) {
      for (int64_t k = in.row_ptr[i]; k < in.row_ptr[i + 1]; ++k) {
        const double v = in.val[k];
        if (v == 0.0) continue;
        rows.idx[rows.start[i] + rows.len[i]] = in.col_idx[k];
        rows.val[rows.start[i] + rows.len[i]] = v;
        ++rows.len[i];
      }
    }
    col_builders.join();
    c = in.c;
    {
      double cmax = 1.0;
      for (double v : c) cmax = std::max(cmax, std::fabs(v));
      cost_tol = kCostTol * cmax;
    }
    off = in.off;
    lo = in.row_lo;
    hi = in.row_hi;
    lx = in.col_lo;
    ux = in.col_hi;
    row_on.assign(m, 1);
    col_on.assign(n, 1);
    dmark_r.assign(m, 0);
    dmark_c.assign(n, 0);
    fixmark.assign(n, 0);
    rmark.assign(m, 0);
  }

  // Run f(lo, hi) over [0, count) on up to 16 threads when count >= min_par
  // (contiguous chunks; f must touch disjoint data per index).
  template <class F>
  static void parallel_for(size_t count, size_t min_par, F f) {
    const unsigned nt = count >= min_par
        ? std::min(16u, std::max(1u, std::thread::hardware_concurrency())) : 1u;
    if (nt <= 1) {
      f((size_t)0, count);
      return;
    }
    ThreadGroup pool;
    for (unsigned t = 0; t < nt; ++t) pool.run(f, count * t / nt, count * (t + 1) / nt);
  }

  void dirty_row(int32_t i) {
    if (!dmark_r[i]) { dmark_r[i] = 1; dlist_r.push_back(i); }
  }
  void dirty_col(int32_t j) {
    if (!dmark_c[j]) { dmark_c[j] = 1; dlist_c.push_back(j); }
  }
  void mark_col_bounds(int32_t j) {
    dirty_col(j);
    for (int32_t q = 0; q < cols.len[j]; ++q) dirty_row(cols.idx[cols.start[j] + q]);
  }
  void remove_entry(int32_t i, int32_t j) {
    rows.erase(i, j);
    cols.erase(j, i);
    dirty_row(i);
    dirty_col(j);
  }
  void set_entry(int32_t i, int32_t j, double v) {
    if (std::fabs(v) < kDropTol) {
      if (rows.find(i, j) >= 0) remove_entry(i, j);
      return;
    }
    rows.put(i, j, v);
    cols.put(j, i, v);
    dirty_row(i);
    dirty_col(j);
  }
  void remove_row(int32_t i) {
    while (rows.len[i] > 0) {
      int32_t j = rows.idx[rows.start[i] + rows.len[i] - 1];
      remove_entry(i, j);
    }
    row_on[i] = 0;
  }
  void remove_col(int32_t j) {
    while (cols.len[j] > 0) {
      int32_t i = cols.idx[cols.start[j] + cols.len[j] - 1];
      remove_entry(i, j);
    }
    col_on[j] = 0;
  }
  void activity(int32_t i, int32_t skip, double &amin, double &amax) const {
    double lo_s = 0.0, hi_s = 0.0;
    int lo_inf = 0, hi_inf = 0;
    int64_t s = rows.start[i];
    for (int32_t q = 0; q < rows.len[i]; ++q) {
      int32_t j = rows.idx[s + q];
      if (j == skip) continue;
      double a = rows.val[s + q];
      double bl, bu;
      if (a > 0) { bl = lx[j]; bu = ux[j]; } else { bl = ux[j]; bu = lx[j]; }
      if (std::isinf(bl)) ++lo_inf; else lo_s += a * bl;
      if (std::isinf(bu)) ++hi_inf; else hi_s += a * bu;
    }
    amin = lo_inf ? -kInf : lo_s;
    amax = hi_inf ? kInf : hi_s;
  }
  PostsolveRecord &push(int32_t kind) {
    PostsolveRecord r{};
    r.kind = kind;
    r.ent_begin = r.ent_end = (int64_t)po->ent_idx.size();
    po->records.push_back(r);
    return po->records.back();
  }
  void push_entry(PostsolveRecord &r, int32_t idx, double v) {
    po->ent_idx.push_back(idx);
    po->ent_val.push_back(v);
    r.ent_end = (int64_t)po->ent_idx.size();
  }

  // ---- rules --------------------------------------------------------------
  void empty_row(int32_t i) {
    if (lo[i] > kFeasTol || hi[i] < -kFeasTol) { status = LP_PRESOLVE_INFEASIBLE; return; }
    PostsolveRecord &r = push(REC_EMPTY_ROW);
    r.i = i;
    row_on[i] = 0;
    po->counts[C_EMPTY_ROW]++;
    changed = true;
  }
  void empty_col(int32_t j) {
    double cj = c[j], v;
    if (cj > cost_tol) v = lx[j];
    else if (cj < -cost_tol) v = ux[j];
    else v = std::min(std::max(0.0, lx[j]), ux[j]);
    if (std::isinf(v)) { status = LP_PRESOLVE_UNBOUNDED; return; }
    off += cj * v;
    PostsolveRecord &r = push(REC_FIX_COL);
    r.j = j; r.v = v; r.cj = cj;
    col_on[j] = 0;
    dirty_col(j);
    po->counts[C_EMPTY_COL]++;
    changed = true;
  }
  void fixed_col(int32_t j) {
    double v = lx[j];
    PostsolveRecord &r = push(REC_FIX_COL);
    r.j = j; r.v = v; r.cj = c[j];
    size_t rec = po->records.size() - 1;
    int64_t s = cols.start[j];
    for (int32_t q = 0; q < cols.len[j]; ++q) {
      int32_t i = cols.idx[s + q];
      double a = cols.val[s + q];
      if (!std::isinf(lo[i])) lo[i] -= a * v;
      if (!std::isinf(hi[i])) hi[i] -= a * v;
      dirty_row(i);
      push_entry(po->records[rec], i, a);
    }
    off += c[j] * v;
    remove_col(j);
    po->counts[C_FIXED_COL]++;
    changed = true;
  }
  // The fixed-column pass as one batch, with the result of one fixed_col
  // call per column in increasing order: fixing x_j changes row bounds and
  // removes column j only, so no decision depends on another; each row's
  // bounds receive the same subtractions in the same (increasing column)
  // order; each touched row is compacted once instead of one erase per entry.
  void fixed_cols(const std::vector<int32_t> &cand) {
    std::vector<int32_t> fx;
    for (int32_t j : cand)
      if (col_on[j] && lx[j] == ux[j]) fx.push_back(j);
    if (fx.size() < 256) {
      for (int32_t j : fx) fixed_col(j);
      return;
    }
    std::vector<int32_t> touched;
    for (int32_t j : fx) {
      const double v = lx[j];
      {
        PostsolveRecord &r = push(REC_FIX_COL);
        r.j = j; r.v = v; r.cj = c[j];
      }
      const size_t rec = po->records.size() - 1;
      const int64_t s = cols.start[j];
      for (int32_t q = 0; q < cols.len[j]; ++q) {
        const int32_t i = cols.idx[s + q];
        push_entry(po->records[rec], i, cols.val[s + q]);
        if (!rmark[i]) { rmark[i] = 1; touched.push_back(i); }
      }
      off += c[j] * v;
      fixmark[j] = 1;
      cols.len[j] = 0;
      col_on[j] = 0;
      dirty_col(j);
      po->counts[C_FIXED_COL]++;
    }
    changed = true;
    parallel_for(touched.size(), 4096, [&](size_t a, size_t b) {
      for (size_t t = a; t < b; ++t) {
        const int32_t i = touched[t];
        const int64_t s = rows.start[i];
        int32_t w = 0;
        double l = lo[i], h = hi[i];
        const bool lf = !std::isinf(l), hf = !std::isinf(h);
        for (int32_t q = 0; q < rows.len[i]; ++q) {
          const int32_t j = rows.idx[s + q];
          const double a = rows.val[s + q];
          if (fixmark[j]) {
            const double v = lx[j];
            if (lf) l -= a * v;
            if (hf) h -= a * v;
          } else {
            rows.idx[s + w] = j;
            rows.val[s + w] = a;
            ++w;
          }
        }
        lo[i] = l;
        hi[i] = h;
        rows.len[i] = w;
        rmark[i] = 0;
      }
    });
    for (int32_t i : touched) dirty_row(i);
    for (int32_t j : fx) fixmark[j] = 0;
  }
  void singleton_row(int32_t i) {
    int32_t j = rows.idx[rows.start[i]];
    double a = rows.val[rows.start[i]];
    double ilo, ihi;
    if (a > 0) {
      ilo = std::isinf(lo[i]) ? -kInf : lo[i] / a;
      ihi = std::isinf(hi[i]) ? kInf : hi[i] / a;
    } else {
      ilo = std::isinf(hi[i]) ? -kInf : hi[i] / a;
      ihi = std::isinf(lo[i]) ? kInf : lo[i] / a;
    }
    bool lo_from = ilo > lx[j];
    bool hi_from = ihi < ux[j];
    double nl = lo_from ? ilo : lx[j];
    double nu = hi_from ? ihi : ux[j];
    if (nl > nu + kFeasTol) { status = LP_PRESOLVE_INFEASIBLE; return; }
    if (nl > nu) nl = nu = 0.5 * (nl + nu);
    PostsolveRecord &r = push(REC_SINGLETON_ROW);
    r.i = i; r.j = j; r.a = a; r.flags = (lo_from ? 1 : 0) | (hi_from ? 2 : 0);
    remove_row(i);
    if (nl != lx[j] || nu != ux[j]) {
      lx[j] = nl;
      ux[j] = nu;
      mark_col_bounds(j);
    }
    po->counts[C_SINGLETON_ROW]++;
    changed = true;
  }
  // redundant rows / dominated sides: the decision for row i given its
  // activity bounds
  void redundant_row_with(int32_t i, double amin, double amax) {
    double l = lo[i], h = hi[i];
    if (l == h) return;
    bool lo_imp = std::isinf(l) || amin >= l;
    bool hi_imp = std::isinf(h) || amax <= h;
    if (lo_imp && hi_imp) {
      PostsolveRecord &r = push(REC_REDUNDANT_ROW);
      r.i = i;
      remove_row(i);
      po->counts[C_REDUNDANT_ROW]++;
      changed = true;
    } else if (lo_imp && !std::isinf(l)) {
      PostsolveRecord &r = push(REC_DROP_SIDE);
      r.i = i; r.flags = 0; r.v = l;
      lo[i] = -kInf;
      dirty_row(i);
      po->counts[C_DROPPED_SIDE]++;
      changed = true;
    } else if (hi_imp && !std::isinf(h)) {
      PostsolveRecord &r = push(REC_DROP_SIDE);
      r.i = i; r.flags = 1; r.v = h;
      hi[i] = kInf;
      dirty_row(i);
      po->counts[C_DROPPED_SIDE]++;
      changed = true;
    }
  }
  void doubleton(int32_t i) {
    int64_t s = rows.start[i];
    int32_t p = rows.idx[s], q = rows.idx[s + 1];
    double ap = rows.val[s], aq = rows.val[s + 1];
    double b = lo[i];
    int32_t j, k;
    double aj, ak;
    if (std::fabs(ap) > std::fabs(aq)) { j = p; aj = ap; k = q; ak = aq; }
    else if (std::fabs(aq) > std::fabs(ap)) { j = q; aj = aq; k = p; ak = ap; }
    else if (cols.len[q] < cols.len[p]) { j = q; aj = aq; k = p; ak = ap; }
    else { j = p; aj = ap; k = q; ak = aq; }
    double r = ak / aj;
    double sv = b / aj;
    double t_lo = std::isinf(ux[j]) ? -kInf : sv - ux[j];
    double t_hi = std::isinf(lx[j]) ? kInf : sv - lx[j];
    double ilo, ihi;
    if (r > 0) {
      ilo = std::isinf(t_lo) ? -kInf : t_lo / r;
      ihi = std::isinf(t_hi) ? kInf : t_hi / r;
    } else {
      ilo = std::isinf(t_hi) ? -kInf : t_hi / r;
      ihi = std::isinf(t_lo) ? kInf : t_lo / r;
    }
    bool lo_from = ilo > lx[k];
    bool hi_from = ihi < ux[k];
    double nl = lo_from ? ilo : lx[k];
    double nu = hi_from ? ihi : ux[k];
    if (nl > nu + kFeasTol) { status = LP_PRESOLVE_INFEASIBLE; return; }
    if (nl > nu) nl = nu = 0.5 * (nl + nu);
    double cj = c[j];
    {
      PostsolveRecord &rec = push(REC_DOUBLETON);
      rec.i = i; rec.j = j; rec.k = k; rec.a = aj; rec.ak = ak; rec.b = b; rec.cj = cj;
      rec.flags = (lo_from ? 1 : 0) | (hi_from ? 2 : 0);
    }
    size_t ri = po->records.size() - 1;
    // snapshot column j without row i (ascending rows)
    std::vector<int32_t> crow;
    std::vector<double> cval;
    int64_t cs = cols.start[j];
    for (int32_t qq = 0; qq < cols.len[j]; ++qq) {
      int32_t rr = cols.idx[cs + qq];
      if (rr == i) continue;
      crow.push_back(rr);
      cval.push_back(cols.val[cs + qq]);
      push_entry(po->records[ri], rr, cols.val[cs + qq]);
    }
    off += cj * sv;
    if (cj != 0.0) {
      c[k] -= cj * r;
      dirty_col(k);
    }
    for (size_t t = 0; t < crow.size(); ++t) {
      int32_t rr = crow[t];
      double a = cval[t];
      if (!std::isinf(lo[rr])) lo[rr] -= a * sv;
      if (!std::isinf(hi[rr])) hi[rr] -= a * sv;
      double old = rows.get(rr, k, 0.0);
      // column j goes as a whole below: drop (rr, j) from the row store only
      rows.erase(rr, j);
      dirty_row(rr);
      set_entry(rr, k, old - a * r);
    }
    cols.len[j] = 0;
    remove_row(i);
    remove_col(j);
    if (nl != lx[k] || nu != ux[k]) {
      lx[k] = nl;
      ux[k] = nu;
      mark_col_bounds(k);
    }
    po->counts[C_DOUBLETON]++;
    changed = true;
  }
  // A row holding x_j up-locks it when a_ij > 0 and its upper side is
  // finite or a_ij < 0 and its lower side is; down-locks mirror that.
  // Whether x_j has a lock in one direction (up: increasing x_j), stopping at
  // the first row that locks it.
  bool locked(int32_t j, bool up) const {
    const int64_t s = cols.start[j];
    for (int32_t q = 0; q < cols.len[j]; ++q) {
      const int32_t i = cols.idx[s + q];
      const bool pos = cols.val[s + q] > 0;
      // up-lock: a > 0 with a finite upper side, a < 0 with a finite lower
      const double side = (pos == up) ? hi[i] : lo[i];
      if (!std::isinf(side)) return true;
    }
    return false;
  }
  // weak dual fixing: c_j < 0 without an up-lock puts x_j at its upper bound
  // in every optimum (z_j < 0), c_j > 0 without a down-lock at its lower
  // bound; the fixed-column reduction does the rest
  void dual_fix(int32_t j) {
    const double cj = c[j];
    if (std::fabs(cj) <= cost_tol) return;
    // c_j < 0 needs no up-lock, c_j > 0 no down-lock
    if (locked(j, cj < 0)) return;
    const double v = cj < 0 ? ux[j] : lx[j];
    if (std::isinf(v)) {
      status = LP_PRESOLVE_UNBOUNDED;
      return;
    }
    lx[j] = v;
    ux[j] = v;
    fixed_col(j);
    po->counts[C_FIXED_COL]--;
    po->counts[C_DUAL_FIX]++;
  }
  void free_col_singleton(int32_t j) {
    int32_t i = cols.idx[cols.start[j]];
    double a = cols.val[cols.start[j]];
    if (!row_on[i] || lo[i] != hi[i] || rows.len[i] < 2) return;
    double b = lo[i];
    bool is_free = std::isinf(lx[j]) && std::isinf(ux[j]);
    if (!is_free) {
      double amin, amax, ilo, ihi;
      activity(i, j, amin, amax);
      if (a > 0) { ilo = (b - amax) / a; ihi = (b - amin) / a; }
      else { ilo = (b - amin) / a; ihi = (b - amax) / a; }
      if (!(ilo >= lx[j] && ihi <= ux[j])) return;
    }
    double cj = c[j];
    {
      PostsolveRecord &rec = push(REC_FREE_COL);
      rec.i = i; rec.j = j; rec.a = a; rec.b = b; rec.cj = cj;
    }
    size_t ri = po->records.size() - 1;
    int64_t s = rows.start[i];
    for (int32_t q = 0; q < rows.len[i]; ++q) {
      int32_t r = rows.idx[s + q];
      if (r == j) continue;
      push_entry(po->records[ri], r, rows.val[s + q]);
    }
    off += cj * b / a;
    if (cj != 0.0) {
      const PostsolveRecord &rec = po->records[ri];
      for (int64_t e = rec.ent_begin; e < rec.ent_end; ++e) {
        int32_t r = po->ent_idx[e];
        c[r] -= cj * po->ent_val[e] / a;
        dirty_col(r);
      }
    }
    remove_row(i);
    remove_col(j);
    po->counts[C_FREE_COL]++;
    changed = true;
  }

  // Column singleton x_j in the inequality row i (Table 1, dual).  Column
  // j's dual constraint a y_i = c_j - z_j, with z_j >= 0 (only l_j finite),
  // <= 0 (only u_j finite) or = 0 (free), bounds y_i on one side of
  // q = c_j / a; y_i >= q > 0 puts every optimum on the row's lower side,
  // y_i <= q < 0 on its upper side, and the row becomes that equality.
  void col_singleton_ineq(int32_t j) {
    const int32_t i = cols.idx[cols.start[j]];
    const double a = cols.val[cols.start[j]];
    if (lo[i] == hi[i]) return;
    const bool lf = !std::isinf(lx[j]), uf = !std::isinf(ux[j]);
    if ((lf && uf) || std::fabs(c[j]) <= cost_tol) return;
    bool y_ge_q, y_le_q;
    if (lf) { y_ge_q = a < 0; y_le_q = a > 0; }
    else if (uf) { y_ge_q = a > 0; y_le_q = a < 0; }
    else { y_ge_q = y_le_q = true; }
    const double q = c[j] / a;
    int side;
    if (y_ge_q && q > 0 && !std::isinf(lo[i])) {
      side = 1;
      hi[i] = lo[i];
    } else if (y_le_q && q < 0 && !std::isinf(hi[i])) {
      side = -1;
      lo[i] = hi[i];
    } else {
      return;
    }
    {
      PostsolveRecord &r = push(REC_ROW_TO_EQ);
      r.i = i;
      r.flags = side > 0 ? 1 : 2;
    }
    const size_t ri = po->records.size() - 1;
    const int64_t s = rows.start[i];
    for (int32_t q2 = 0; q2 < rows.len[i]; ++q2)
      push_entry(po->records[ri], rows.idx[s + q2], rows.val[s + q2]);
    dirty_row(i);
    po->counts[C_INEQ_TO_EQ]++;
    changed = true;
  }
  bool same_pattern(int32_t i, int32_t k) const {
    if (rows.len[i] != rows.len[k]) return false;
    return std::memcmp(&rows.idx[rows.start[i]], &rows.idx[rows.start[k]],
                       sizeof(int32_t) * rows.len[i]) == 0;
  }
  // s with a_k = s a_i to kParTol (same pattern), s taken at the first column
  bool parallel_scale(int32_t i, int32_t k, double &s) const {
    const double *vi = &rows.val[rows.start[i]];
    const double *vk = &rows.val[rows.start[k]];
    s = vk[0] / vi[0];
    for (int32_t q = 0; q < rows.len[i]; ++q)
      if (std::fabs(vk[q] - s * vi[q]) > kParTol * std::fabs(vk[q])) return false;
    return true;
  }
  void merge_parallel(int32_t i, int32_t k, double s) {
    const double lk = lo[k], uk = hi[k];
    double nlk, nuk;
    if (s > 0) {
      nlk = std::isinf(lk) ? -kInf : lk / s;
      nuk = std::isinf(uk) ? kInf : uk / s;
    } else {
      nlk = std::isinf(uk) ? -kInf : uk / s;
      nuk = std::isinf(lk) ? kInf : lk / s;
    }
    const bool lo_from = nlk > lo[i];
    const bool hi_from = nuk < hi[i];
    double nl = lo_from ? nlk : lo[i];
    double nu = hi_from ? nuk : hi[i];
    if (nl > nu + kFeasTol) { status = LP_PRESOLVE_INFEASIBLE; return; }
    if (nl > nu) nl = nu = 0.5 * (nl + nu);
    PostsolveRecord &r = push(REC_PARALLEL_ROW);
    r.i = i; r.k = k; r.a = s; r.flags = (lo_from ? 1 : 0) | (hi_from ? 2 : 0);
    remove_row(k);
    if (nl != lo[i] || nu != hi[i]) {
      lo[i] = nl;
      hi[i] = nu;
      dirty_row(i);
    }
    po->counts[C_PARALLEL_ROW]++;
    changed = true;
  }
  // Medium explorer (Table 1): rows grouped by a hash of their column
  // pattern; within a hash group, in increasing index, a row is merged into
  // the first of the first kParCandidates earlier unmerged rows of the same
  // pattern that it is parallel to.  The test reads coefficients only, so
  // all merges are found first and applied in increasing row order.
  void parallel_rows() {
    std::vector<std::pair<uint64_t, int32_t>> key;
    for (int32_t i = 0; i < m; ++i)
      if (row_on[i] && rows.len[i] >= 2) key.emplace_back(0, i);
    parallel_for(key.size(), 20000, [&](size_t a, size_t b) {
      for (size_t t = a; t < b; ++t) {
        const int32_t i = key[t].second;
        uint64_t h = 1469598103934665603ull ^ (uint64_t)rows.len[i];
        const int64_t s = rows.start[i];
        for (int32_t q = 0; q < rows.len[i]; ++q) {
          h ^= (uint64_t)(uint32_t)rows.idx[s + q];
          h *= 1099511628211ull;
        }
        key[t].first = h;
      }
    });
    std::sort(key.begin(), key.end());
    struct Merge { int32_t k, i; double s; };
    std::vector<Merge> merges;
    std::vector<int32_t> reps;
    for (size_t a = 0; a < key.size();) {
      size_t b = a + 1;
      while (b < key.size() && key[b].first == key[a].first) ++b;
      if (b - a > 1) {
        reps.clear();
        for (size_t t = a; t < b; ++t) {
          const int32_t k = key[t].second;
          int found = -1, checked = 0;
          double s = 0.0;
          for (int32_t i : reps) {
            if (!same_pattern(i, k)) continue;
            if (checked++ >= kParCandidates) break;
            if (parallel_scale(i, k, s)) { found = i; break; }
          }
          if (found >= 0) merges.push_back({k, found, s});
          else reps.push_back(k);
        }
      }
      a = b;
    }
    std::sort(merges.begin(), merges.end(),
              [](const Merge &x, const Merge &y) { return x.k < y.k; });
    for (const Merge &g : merges) {
      merge_parallel(g.i, g.k, g.s);
      if (status != LP_PRESOLVE_REDUCED) return;
    }
  }

  // Primal propagation (Table 1, medium; enabled by LP_RULE_PRIMAL_PROPAGATION).
  // From row i's activity bounds at the start of the row (finite
  // contributions summed in increasing column order, infinite ones counted;
  // a column's "others" bound is the total minus its own finite part, or the
  // total when its own part is the only infinite one): a_ij x_j >= l_i -
  // max(others), a_ij x_j <= u_i - min(others).
  static bool prop_better(double nw, double old, bool lower) {
    if (std::isinf(nw)) return false;
    if (std::isinf(old)) return std::fabs(nw) <= kPropMaxBound;
    const double step = kPropStep * std::max(1.0, std::fabs(old));
    return lower ? nw > old + step : nw < old - step;
  }
  void propagate_row(int32_t i) {
    const double lo_i = lo[i], hi_i = hi[i];
    const int64_t s = rows.start[i];
    const int32_t len = rows.len[i];
    double smin = 0.0, smax = 0.0;
    int nmin = 0, nmax = 0;
    for (int32_t q = 0; q < len; ++q) {
      const int32_t j = rows.idx[s + q];
      const double a = rows.val[s + q];
      const double bl = a > 0 ? lx[j] : ux[j], bu = a > 0 ? ux[j] : lx[j];
      if (std::isinf(bl)) ++nmin; else smin += a * bl;
      if (std::isinf(bu)) ++nmax; else smax += a * bu;
    }
    if ((int32_t)prop_lo.size() < len) {
      prop_lo.resize(len);
      prop_hi.resize(len);
    }
    double *nls = prop_lo.data(), *nus = prop_hi.data();
    for (int32_t q = 0; q < len; ++q) {
      const int32_t j = rows.idx[s + q];
      const double a = rows.val[s + q];
      const double bl = a > 0 ? lx[j] : ux[j], bu = a > 0 ? ux[j] : lx[j];
      const double omax = std::isinf(bu) ? (nmax == 1 ? smax : kInf) : (nmax == 0 ? smax - a * bu : kInf);
      const double omin = std::isinf(bl) ? (nmin == 1 ? smin : -kInf) : (nmin == 0 ? smin - a * bl : -kInf);
      const double t_lo = (!std::isinf(lo_i) && !std::isinf(omax)) ? lo_i - omax : -kInf;
      const double t_hi = (!std::isinf(hi_i) && !std::isinf(omin)) ? hi_i - omin : kInf;
      if (a > 0) {
        nls[q] = std::isinf(t_lo) ? -kInf : t_lo / a;
        nus[q] = std::isinf(t_hi) ? kInf : t_hi / a;
      } else {
        nls[q] = std::isinf(t_hi) ? -kInf : t_hi / a;
        nus[q] = std::isinf(t_lo) ? kInf : t_lo / a;
      }
    }
    for (int32_t q = 0; q < len; ++q) {
      const int32_t j = rows.idx[s + q];
      const double a = rows.val[s + q];
      for (int side = 0; side < 2; ++side) {
        double nw = side == 0 ? nls[q] : nus[q];
        const double old = side == 0 ? lx[j] : ux[j];
        if (!prop_better(nw, old, side == 0)) continue;
        const double other = side == 0 ? ux[j] : lx[j];
        if (side == 0 ? nw > other + kFeasTol : nw < other - kFeasTol) {
          status = LP_PRESOLVE_INFEASIBLE;
          return;
        }
        if (side == 0 ? nw > other : nw < other) nw = other;
        {
          PostsolveRecord &r = push(REC_TIGHTEN);
          r.j = j; r.i = i; r.a = a; r.flags = side;
        }
        const size_t ri = po->records.size() - 1;
        for (int32_t q2 = 0; q2 < len; ++q2)
          push_entry(po->records[ri], rows.idx[s + q2], rows.val[s + q2]);
        if (side == 0) lx[j] = nw; else ux[j] = nw;
        mark_col_bounds(j);
        po->counts[C_TIGHTENED]++;
        changed = true;
      }
    }
  }
  void propagate() {
    for (int32_t i = 0; i < m; ++i)
      if (row_on[i] && rows.len[i] >= 2) {
        propagate_row(i);
        if (status != LP_PRESOLVE_REDUCED) return;
      }
  }

  // Dual propagation (Table 1, medium; enabled by LP_RULE_DUAL_PROPAGATION):
  // one sweep of dual bounds.  Rows start from the sign domain of y_i; each
  // column j with x_j not boxed bounds S_j = sum_i a_ij y_i by c_j - z_j with
  // z_j's sign domain, and its rows (ascending) get the bounds S_j minus the
  // others' dual activity implies (from the bounds at the start of the
  // column).  Rows whose dual is bounded away from 0 become equalities, then
  // columns whose reduced cost is are fixed (dual reductions).
  static void scaled_range(double a, double lo, double hi, double &rlo, double &rhi) {
    if (a > 0) {
      rlo = std::isinf(lo) ? -kInf : a * lo;
      rhi = std::isinf(hi) ? kInf : a * hi;
    } else {
      rlo = std::isinf(hi) ? -kInf : a * hi;
      rhi = std::isinf(lo) ? kInf : a * lo;
    }
  }
  void dual_propagate() {
    std::vector<double> yl(m, -kInf), yu(m, kInf);
    for (int32_t i = 0; i < m; ++i)
      if (row_on[i]) {
        yl[i] = std::isinf(hi[i]) ? 0.0 : -kInf;
        yu[i] = std::isinf(lo[i]) ? 0.0 : kInf;
      }
    std::vector<double> tlo, thi, nls, nus;
    for (int32_t j = 0; j < n; ++j) {
      if (!col_on[j] || cols.len[j] == 0) continue;
      const bool lf = !std::isinf(lx[j]), uf = !std::isinf(ux[j]);
      if (lf && uf) continue;
      const double cj = c[j];
      const double dl = lf ? -kInf : cj, du = uf ? kInf : cj;
      const int64_t s0 = cols.start[j];
      const int32_t len = cols.len[j];
      tlo.resize(len);
      thi.resize(len);
      nls.resize(len);
      nus.resize(len);
      double slo = 0.0, shi = 0.0;
      int nlo = 0, nhi = 0;
      for (int32_t q = 0; q < len; ++q) {
        const int32_t i = cols.idx[s0 + q];
        scaled_range(cols.val[s0 + q], yl[i], yu[i], tlo[q], thi[q]);
        if (std::isinf(tlo[q])) ++nlo; else slo += tlo[q];
        if (std::isinf(thi[q])) ++nhi; else shi += thi[q];
      }
      for (int32_t q = 0; q < len; ++q) {
        const double a = cols.val[s0 + q];
        const double omax = std::isinf(thi[q]) ? (nhi == 1 ? shi : kInf)
                                               : (nhi == 0 ? shi - thi[q] : kInf);
        const double omin = std::isinf(tlo[q]) ? (nlo == 1 ? slo : -kInf)
                                               : (nlo == 0 ? slo - tlo[q] : -kInf);
        const double t_lo = (!std::isinf(dl) && !std::isinf(omax)) ? dl - omax : -kInf;
        const double t_hi = (!std::isinf(du) && !std::isinf(omin)) ? du - omin : kInf;
        if (a > 0) {
          nls[q] = std::isinf(t_lo) ? -kInf : t_lo / a;
          nus[q] = std::isinf(t_hi) ? kInf : t_hi / a;
        } else {
          nls[q] = std::isinf(t_hi) ? -kInf : t_hi / a;
          nus[q] = std::isinf(t_lo) ? kInf : t_lo / a;
        }
      }
      for (int32_t q = 0; q < len; ++q) {
        const int32_t i = cols.idx[s0 + q];
        if (nls[q] > yl[i]) yl[i] = nls[q];
        if (nus[q] < yu[i]) yu[i] = nus[q];
      }
    }
    for (int32_t i = 0; i < m; ++i) {
      if (!row_on[i] || lo[i] == hi[i] || rows.len[i] == 0) continue;
      int side;
      if (yl[i] >= kDualPropTol && !std::isinf(lo[i])) {
        side = 1;
        hi[i] = lo[i];
      } else if (yu[i] <= -kDualPropTol && !std::isinf(hi[i])) {
        side = -1;
        lo[i] = hi[i];
      } else {
        continue;
      }
      {
        PostsolveRecord &r = push(REC_ROW_TO_EQ);
        r.i = i;
        r.flags = side > 0 ? 1 : 2;
      }
      const size_t ri = po->records.size() - 1;
      const int64_t s = rows.start[i];
      for (int32_t q = 0; q < rows.len[i]; ++q)
        push_entry(po->records[ri], rows.idx[s + q], rows.val[s + q]);
      dirty_row(i);
      po->counts[C_DUAL_PROP]++;
      changed = true;
    }
    for (int32_t j = 0; j < n; ++j) {
      if (!col_on[j] || cols.len[j] == 0 || lx[j] == ux[j]) continue;
      const int64_t s0 = cols.start[j];
      double slo = 0.0, shi = 0.0;
      int nlo = 0, nhi = 0;
      for (int32_t q = 0; q < cols.len[j]; ++q) {
        const int32_t i = cols.idx[s0 + q];
        double rlo, rhi;
        scaled_range(cols.val[s0 + q], yl[i], yu[i], rlo, rhi);
        if (std::isinf(rlo)) ++nlo; else slo += rlo;
        if (std::isinf(rhi)) ++nhi; else shi += rhi;
      }
      const double cj = c[j];
      const double tol = kDualPropTol * std::max(1.0, std::fabs(cj));
      const double zmin = nhi == 0 ? cj - shi : -kInf;
      const double zmax = nlo == 0 ? cj - slo : kInf;
      double v;
      if (zmin > tol && !std::isinf(lx[j])) v = lx[j];
      else if (zmax < -tol && !std::isinf(ux[j])) v = ux[j];
      else continue;
      lx[j] = v;
      ux[j] = v;
      fixed_col(j);
      po->counts[C_FIXED_COL]--;
      po->counts[C_DUAL_PROP]++;
    }
  }

  // Parallel columns (Table 1, medium; enabled by LP_RULE_PARALLEL_COLS):
  // the column analogue of parallel_rows, with the costs parallel as well.
  bool same_col_pattern(int32_t j, int32_t k) const {
    if (cols.len[j] != cols.len[k]) return false;
    return std::memcmp(&cols.idx[cols.start[j]], &cols.idx[cols.start[k]],
                       sizeof(int32_t) * cols.len[j]) == 0;
  }
  bool parallel_col_scale(int32_t j, int32_t k, double &s) const {
    const double *vj = &cols.val[cols.start[j]];
    const double *vk = &cols.val[cols.start[k]];
    s = vk[0] / vj[0];
    for (int32_t q = 0; q < cols.len[j]; ++q)
      if (std::fabs(vk[q] - s * vj[q]) > kParTol * std::fabs(vk[q])) return false;
    const double sc = s * c[j];
    return !(std::fabs(c[k] - sc) > kParTol * std::max(std::fabs(c[k]), std::fabs(sc)));
  }
  void merge_parallel_col(int32_t j, int32_t k, double s) {
    const double lj = lx[j], uj = ux[j], lk = lx[k], uk = ux[k];
    double nl, nu;
    if (s > 0) { nl = lj + s * lk; nu = uj + s * uk; }
    else { nl = lj + s * uk; nu = uj + s * lk; }
    {
      // the record's b, cj, v, ak hold l_j, u_j, l_k, u_k
      PostsolveRecord &r = push(REC_PARALLEL_COL);
      r.j = j; r.k = k; r.a = s; r.b = lj; r.cj = uj; r.v = lk; r.ak = uk;
    }
    remove_col(k);
    lx[j] = nl;
    ux[j] = nu;
    mark_col_bounds(j);
    po->counts[C_PARALLEL_COL]++;
    changed = true;
  }
  void parallel_cols() {
    std::vector<std::pair<uint64_t, int32_t>> key;
    for (int32_t j = 0; j < n; ++j)
      if (col_on[j] && cols.len[j] >= 2) key.emplace_back(0, j);
    parallel_for(key.size(), 20000, [&](size_t a, size_t b) {
      for (size_t t = a; t < b; ++t) {
        const int32_t j = key[t].second;
        uint64_t h = 1469598103934665603ull ^ (uint64_t)cols.len[j];
        const int64_t s = cols.start[j];
        for (int32_t q = 0; q < cols.len[j]; ++q) {
          h ^= (uint64_t)(uint32_t)cols.idx[s + q];
          h *= 1099511628211ull;
        }
        key[t].first = h;
      }
    });
    std::sort(key.begin(), key.end());
    struct Merge { int32_t k, j; double s; };
    std::vector<Merge> merges;
    std::vector<int32_t> reps;
    for (size_t a = 0; a < key.size();) {
      size_t b = a + 1;
      while (b < key.size() && key[b].first == key[a].first) ++b;
      if (b - a > 1) {
        reps.clear();
        for (size_t t = a; t < b; ++t) {
          const int32_t k = key[t].second;
          int found = -1, checked = 0;
          double s = 0.0;
          for (int32_t j : reps) {
            if (!same_col_pattern(j, k)) continue;
            if (checked++ >= kParCandidates) break;
            if (parallel_col_scale(j, k, s)) { found = j; break; }
          }
          if (found >= 0) merges.push_back({k, found, s});
          else reps.push_back(k);
        }
      }
      a = b;
    }
    std::sort(merges.begin(), merges.end(),
              [](const Merge &x, const Merge &y) { return x.k < y.k; });
    for (const Merge &g : merges) merge_parallel_col(g.j, g.k, g.s);
  }

  int run(int max_rounds, int mask) {
    int prop_sweeps = 0, dual_sweeps = 0;
    std::vector<int32_t> rc(m), cc(n);
    for (int32_t i = 0; i < m; ++i) rc[i] = i;
    for (int32_t j = 0; j < n; ++j) cc[j] = j;
    int rounds = 0;
    for (int rnd = 0; rnd < max_rounds; ++rnd) {
      rounds = rnd + 1;
      for (int32_t i : dlist_r) dmark_r[i] = 0;
      for (int32_t j : dlist_c) dmark_c[j] = 0;
      dlist_r.clear();
      dlist_c.clear();
      changed = false;
      if (mask & LP_RULE_EMPTY_ROW)
        for (int32_t i : rc)
          if (row_on[i] && rows.len[i] == 0) {
            empty_row(i);
            if (status != LP_PRESOLVE_REDUCED) return rounds;
          }
      if (mask & LP_RULE_EMPTY_COL)
        for (int32_t j : cc)
          if (col_on[j] && cols.len[j] == 0) {
            empty_col(j);
            if (status != LP_PRESOLVE_REDUCED) return rounds;
          }
      if (mask & LP_RULE_FIXED_COL) fixed_cols(cc);
      if (mask & LP_RULE_SINGLETON_ROW)
        for (int32_t i : rc)
          if (row_on[i] && rows.len[i] == 1) {
            singleton_row(i);
            if (status != LP_PRESOLVE_REDUCED) return rounds;
          }
      if (mask & LP_RULE_REDUNDANT_ROW) {
        // The pass changes no column bound and no other row's entries, so
        // every candidate's activity bounds can be computed first (in
        // parallel for large candidate sets, each a sequential sum in the
        // same order), then the decisions applied in index order.
        std::vector<int32_t> cand;
        for (int32_t i : rc)
          if (row_on[i] && rows.len[i] >= 1 && lo[i] != hi[i]) cand.push_back(i);
        std::vector<double> amin(cand.size()), amax(cand.size());
        const size_t nc = cand.size();
        parallel_for(nc, 20000, [&](size_t a, size_t b) {
          for (size_t q = a; q < b; ++q) activity(cand[q], -1, amin[q], amax[q]);
        });
        for (size_t q = 0; q < nc; ++q) redundant_row_with(cand[q], amin[q], amax[q]);
      }
      if (mask & LP_RULE_DOUBLETON)
        for (int32_t i : rc)
          if (row_on[i] && rows.len[i] == 2 && lo[i] == hi[i]) {
            doubleton(i);
            if (status != LP_PRESOLVE_REDUCED) return rounds;
          }
      if (mask & LP_RULE_COL_SINGLETON_INEQ)
        for (int32_t j : cc)
          if (col_on[j] && cols.len[j] == 1) col_singleton_ineq(j);
      if (mask & LP_RULE_FREE_COL_SINGLETON)
        for (int32_t j : cc)
          if (col_on[j] && cols.len[j] == 1) free_col_singleton(j);
      if (mask & LP_RULE_VARIABLE_LOCKS)
        for (int32_t j : cc)
          if (col_on[j] && cols.len[j] > 0) {
            dual_fix(j);
            if (status != LP_PRESOLVE_REDUCED) return rounds;
          }
      if (!changed) {
        if ((mask & LP_RULE_PRIMAL_PROPAGATION) && prop_sweeps < kPropSweeps) {
          ++prop_sweeps;
          propagate();
          if (status != LP_PRESOLVE_REDUCED) return rounds;
        }
        if ((mask & LP_RULE_DUAL_PROPAGATION) && dual_sweeps < 1) {
          ++dual_sweeps;
          dual_propagate();
        }
        if (mask & LP_RULE_PARALLEL_ROWS) {
          parallel_rows();
          if (status != LP_PRESOLVE_REDUCED) return rounds;
        }
        if (mask & LP_RULE_PARALLEL_COLS) parallel_cols();
        if (!changed) break;
      }
      rc.clear();
      cc.clear();
      for (int32_t i : dlist_r) if (row_on[i]) rc.push_back(i);
      for (int32_t j : dlist_c) if (col_on[j]) cc.push_back(j);
      std::sort(rc.begin(), rc.end());
      std::sort(cc.begin(), cc.end());
    }
    return rounds;
  }

  void build_reduced(HostLP &out) {
    po->row_map.clear();
    po->col_map.clear();
    std::vector<int32_t> cpos(n, -1);
    for (int32_t j = 0; j < n; ++j)
      if (col_on[j]) { cpos[j] = (int32_t)po->col_map.size(); po->col_map.push_back(j); }
    for (int32_t i = 0; i < m; ++i)
      if (row_on[i]) po->row_map.push_back(i);
    out = HostLP();
    out.m = (int32_t)po->row_map.size();
    out.n = (int32_t)po->col_map.size();
    out.row_ptr.assign(out.m + 1, 0);
    for (int32_t r = 0; r < out.m; ++r) out.row_ptr[r + 1] = out.row_ptr[r] + rows.len[po->row_map[r]];
    const int64_t nz = out.row_ptr[out.m];
    out.col_idx.resize(nz);
    out.val.resize(nz);
    out.row_lo.resize(out.m);
    out.row_hi.resize(out.m);
    parallel_for((size_t)out.m, 20000, [&](size_t a, size_t b) {
      for (size_t r = a; r < b; ++r) {
        const int32_t i = po->row_map[r];
        const int64_t s = rows.start[i];
        int64_t w = out.row_ptr[r];
        for (int32_t q = 0; q < rows.len[i]; ++q, ++w) {
          out.col_idx[w] = cpos[rows.idx[s + q]];
          out.val[w] = rows.val[s + q];
        }
        out.row_lo[r] = lo[i];
        out.row_hi[r] = hi[i];
      }
    });
    for (int32_t j : po->col_map) {
      out.c.push_back(c[j]);
      out.col_lo.push_back(lx[j]);
      out.col_hi.push_back(ux[j]);
    }
    out.off = off;
  }
};

}  // namespace

void presolve_run(const HostLP &in, int max_rounds, int rule_mask, HostLP &out,
                  PresolveOutcome &po) {
  po = PresolveOutcome();
  po.m0 = in.m;
  po.n0 = in.n;
  Presolver ps(in, &po);
  po.rounds = ps.run(max_rounds, rule_mask);
  po.status = ps.status;
  ps.build_reduced(out);
  if (po.status == LP_PRESOLVE_REDUCED && out.m == 0 && out.n == 0)
    po.status = LP_PRESOLVE_SOLVED;
}

void postsolve_run(const PresolveOutcome &po, const HostLP &red, const double *xr,
                   const double *yr, const double *zr, double *x, double *y, double *z) {
  std::fill(x, x + po.n0, 0.0);
  std::fill(y, y + po.m0, 0.0);
  std::fill(z, z + po.n0, 0.0);
  for (int32_t q = 0; q < red.n; ++q) x[po.col_map[q]] = xr[q];
  for (int32_t r = 0; r < red.m; ++r) y[po.row_map[r]] = yr[r];
  if (zr) {
    for (int32_t q = 0; q < red.n; ++q) z[po.col_map[q]] = zr[q];
  } else {
    std::vector<double> g(red.c);
    for (int32_t r = 0; r < red.m; ++r)
      for (int64_t e = red.row_ptr[r]; e < red.row_ptr[r + 1]; ++e)
        g[red.col_idx[e]] -= red.val[e] * yr[r];
    for (int32_t q = 0; q < red.n; ++q) z[po.col_map[q]] = g[q];
  }
  for (size_t t = po.records.size(); t-- > 0;) {
    const PostsolveRecord &r = po.records[t];
    switch (r.kind) {
      case REC_EMPTY_ROW:
      case REC_REDUNDANT_ROW:
        y[r.i] = 0.0;
        break;
      case REC_DROP_SIDE:
        break;
      case REC_FIX_COL: {
        x[r.j] = r.v;
        double s = r.cj;
        for (int64_t e = r.ent_begin; e < r.ent_end; ++e) s -= po.ent_val[e] * y[po.ent_idx[e]];
        z[r.j] = s;
        break;
      }
      case REC_SINGLETON_ROW: {
        bool lo_from = r.flags & 1, hi_from = r.flags & 2;
        if ((z[r.j] > 0 && lo_from) || (z[r.j] < 0 && hi_from)) {
          y[r.i] = z[r.j] / r.a;
          z[r.j] = 0.0;
        } else {
          y[r.i] = 0.0;
        }
        break;
      }
      case REC_DOUBLETON: {
        int32_t i = r.i, j = r.j, k = r.k;
        double aj = r.a, ak = r.ak;
        x[j] = (r.b - ak * x[k]) / aj;
        double dj = r.cj;
        for (int64_t e = r.ent_begin; e < r.ent_end; ++e) dj -= po.ent_val[e] * y[po.ent_idx[e]];
        bool lo_from = r.flags & 1, hi_from = r.flags & 2;
        if ((z[k] > 0 && lo_from) || (z[k] < 0 && hi_from)) {
          y[i] = (z[k] + (ak / aj) * dj) / ak;
          z[j] = dj - aj * y[i];
          z[k] = 0.0;
        } else {
          y[i] = dj / aj;
          z[j] = 0.0;
        }
        break;
      }
      case REC_ROW_TO_EQ: {
        if (((r.flags & 1) && y[r.i] < 0) || ((r.flags & 2) && y[r.i] > 0)) {
          const double d = -y[r.i];
          y[r.i] = 0.0;
          for (int64_t e = r.ent_begin; e < r.ent_end; ++e) z[po.ent_idx[e]] -= po.ent_val[e] * d;
        }
        break;
      }
      case REC_TIGHTEN: {
        if ((r.flags == 0 && z[r.j] > 0) || (r.flags == 1 && z[r.j] < 0)) {
          const double d = z[r.j] / r.a;
          y[r.i] += d;
          for (int64_t e = r.ent_begin; e < r.ent_end; ++e) z[po.ent_idx[e]] -= po.ent_val[e] * d;
          z[r.j] = 0.0;
        }
        break;
      }
      case REC_PARALLEL_COL: {
        const double s = r.a, lj = r.b, uj = r.cj, lk = r.v, uk = r.ak;
        const double v = x[r.j];
        double xk = std::min(std::max(0.0, lk), uk);
        double xj = v - s * xk;
        if (xj < lj) {
          xj = lj;
          xk = std::min(std::max((v - xj) / s, lk), uk);
        } else if (xj > uj) {
          xj = uj;
          xk = std::min(std::max((v - xj) / s, lk), uk);
        }
        x[r.j] = xj;
        x[r.k] = xk;
        z[r.k] = s * z[r.j];
        break;
      }
      case REC_PARALLEL_ROW: {
        const bool lo_from = r.flags & 1, hi_from = r.flags & 2;
        if ((y[r.i] > 0 && lo_from) || (y[r.i] < 0 && hi_from)) {
          y[r.k] = y[r.i] / r.a;
          y[r.i] = 0.0;
        } else {
          y[r.k] = 0.0;
        }
        break;
      }
      case REC_FREE_COL: {
        double s = r.b;
        for (int64_t e = r.ent_begin; e < r.ent_end; ++e) s -= po.ent_val[e] * x[po.ent_idx[e]];
        x[r.j] = s / r.a;
        y[r.i] = r.cj / r.a;
        z[r.j] = 0.0;
        break;
      }
      default:
        break;
    }
  }
}

}  // namespace gb300lp
