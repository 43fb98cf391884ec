// C ABI entry points (include/lp.h): validation, host problem storage,
// presolve / postsolve dispatch, and the host rel-KKT measure.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <cstdlib>
#include <cstdio>
#include <exception>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "host_parallel.h"
#include "lp_internal.h"

using namespace gb300lp;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
}  // namespace

namespace gb300lp {
void set_last_error(const std::string &m) { g_err = m; }

void trace_state(const char *engine, long long t, double rel_kkt, double rel_p, double rel_d,
                 double rel_gap, double omega, int restarts, int fp32) {
  static std::mutex mu;
  static bool opened = false;
  static FILE *f = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!opened) {
    opened = true;
    const char *path = std::getenv("LP_TRACE");
    if (path && *path) f = std::fopen(path, "a");
  }
  if (!f) return;
  std::fprintf(f,
               "{\"engine\": \"%s\", \"t\": %lld, \"rel_kkt\": %.6e, \"rel_p\": %.6e, "
               "\"rel_d\": %.6e, \"rel_gap\": %.6e, \"omega\": %.6e, \"restarts\": %d, "
               "\"fp32\": %d}\n",
               engine, t, rel_kkt, rel_p, rel_d, rel_gap, omega, restarts, fp32);
  std::fflush(f);
}
}  // namespace gb300lp

struct lp_problem {
  HostLP orig;
  HostLP cur;
  bool presolved = false;
  PresolveOutcome po;
  bool has_dev = false;
  lp_device_ctx dev{};
  DeviceLP *dlp = nullptr;
  DeviceSolution sol;
  int32_t last_termination = -1;
};

namespace gb300lp {
// used by the batch server (batch.cu) to read a problem's current LP
const HostLP &problem_current(const lp_problem *lp) { return lp->cur; }
// the LP as created: held in `orig` once presolved, else the current one
const HostLP &original_lp(const lp_problem *lp) { return lp->presolved ? lp->orig : lp->cur; }
// LP_INFEASIBLE / LP_UNBOUNDED when the presolve proved it, else -1
int problem_proven_status(const lp_problem *lp) {
  if (!lp->presolved) return -1;
  if (lp->po.status == LP_PRESOLVE_INFEASIBLE) return LP_INFEASIBLE;
  if (lp->po.status == LP_PRESOLVE_UNBOUNDED) return LP_UNBOUNDED;
  return -1;
}
// rel-KKT on the original LP of the postsolved reduced solution (x, y, z of
// the current LP), or -1 when the problem was not presolved (the current LP
// is the original and the device measure already applies to it)
// the measures of host_rel_kkt for the postsolved point on the original LP
// (k[0] = rel-KKT; -1 when the problem was not presolved)
void problem_original_measures(const lp_problem *lp, const double *x, const double *y,
                               const double *z, double k[9]) {
  k[0] = -1.0;
  if (!lp->presolved) return;
  std::vector<double> X(lp->orig.n), Y(lp->orig.m), Z(lp->orig.n);
  postsolve_run(lp->po, lp->cur, x, y, z, X.data(), Y.data(), Z.data());
  host_rel_kkt(lp->orig, X.data(), Y.data(), k);
}
double problem_original_kkt(const lp_problem *lp, const double *x, const double *y,
                            const double *z) {
  double k[9];
  problem_original_measures(lp, x, y, z, k);
  return k[0];
}
void problem_store_solution(lp_problem *lp, const std::vector<double> &x,
                            const std::vector<double> &y, const std::vector<double> &z) {
  lp->sol.x = x;
  lp->sol.y = y;
  lp->sol.z = z;
  lp->sol.xi = x;
  lp->sol.yi = y;
  lp->sol.valid = true;
}
}  // namespace gb300lp

namespace gb300lp {
bool valid_solve_opts(const lp_solve_opts &o) {
  return o.eps_rel >= 0 && o.max_iter >= 1 && o.check_every >= 1 && o.rho >= 0 && o.rho <= 1 &&
         o.infeas_every >= 0 && o.eps_infeas >= 0 &&
         (o.primal_weight_clamp == 0.0 || o.primal_weight_clamp >= 1.0) &&
         (o.precision == LP_FP64 || o.precision == LP_MIXED) && o.engine >= LP_ENGINE_AUTO &&
         o.engine <= LP_ENGINE_CLUSTER && o.refine_original >= 0 && o.refine_original <= 8 &&
         (o.tile_run_max == 0 || o.tile_run_max == 8 || o.tile_run_max == 16 ||
          o.tile_run_max == 32 || o.tile_run_max == 64) &&
         (o.tile_nnz == 0 || o.tile_nnz == 512 || o.tile_nnz == 2048) && o.eps_gap_rel >= 0 &&
         (o.polish == 0 || o.polish == 1) && o.polish_fraction > 0 && o.polish_fraction <= 8 &&
         !(o.polish && o.engine == LP_ENGINE_CLUSTER);
}
}  // namespace gb300lp

#define API_GUARD_BEGIN try {
#define API_GUARD_END                                                   \
  }                                                                     \
  catch (const std::bad_alloc &) {                                      \
    return fail(LP_ERR_OOM, "host allocation failed");                  \
  }                                                                     \
  catch (const std::exception &e) {                                     \
    return fail(LP_ERR_INVALID, std::string("internal error: ") + e.what()); \
  }                                                                     \
  catch (...) {                                                         \
    return fail(LP_ERR_INVALID, "internal error");                      \
  }

extern "C" {

void lp_solve_opts_default(lp_solve_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->infeas_every = 4;
  o->eps_infeas = 1e-8;
  o->primal_weight_clamp = 10.0;
  o->refine_original = 3;
  o->polish_fraction = 0.125;
  o->eps_rel = 1e-6;
  o->max_iter = 200000;
  o->time_limit_s = 3600.0;
  o->precision = LP_FP64;
  o->check_every = 64;
  o->rho = 1.0;
  o->beta_suff = 0.2;
  o->beta_nec = 0.8;
  o->beta_art = 0.36;
  o->theta = 0.5;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->power_iters = 100;
  o->halpern = 1;
  o->restarts = 1;
  o->use_graph = 1;
  o->step_size = 0.0;
  o->primal_weight = 0.0;
  o->x_init = nullptr;
  o->y_init = nullptr;
  o->engine = LP_ENGINE_AUTO;
  o->verbose = 0;
}

void lp_presolve_opts_default(lp_presolve_opts *o) {
  if (!o) return;
  o->max_rounds = 20;
  o->enable = LP_RULE_ALL;
}

const char *lp_last_error(void) { return g_err.c_str(); }

int lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
              const int32_t *col_idx, const double *val, const double *c,
              double obj_offset, const double *row_lo, const double *row_hi,
              const double *col_lo, const double *col_hi, const lp_device_ctx *dev,
              lp_problem **out) {
  API_GUARD_BEGIN
  if (!out) return fail(LP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (m < 0 || n < 0 || nnz < 0) return fail(LP_ERR_INVALID, "negative size");
  if (!row_ptr) return fail(LP_ERR_INVALID, "row_ptr is NULL");
  if (nnz > 0 && (!col_idx || !val)) return fail(LP_ERR_INVALID, "col_idx/val NULL");
  if ((n > 0 && (!c || !col_lo || !col_hi)) || (m > 0 && (!row_lo || !row_hi)))
    return fail(LP_ERR_INVALID, "vector argument is NULL");
  if (row_ptr[0] != 0 || row_ptr[m] != nnz)
    return fail(LP_ERR_INVALID, "row_ptr must start at 0 and end at nnz");
  for (int32_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return fail(LP_ERR_INVALID, "row_ptr decreases");
  {
    // the rows' entries, checked in row chunks on host threads; the first
    // failing row of the first failing chunk gives the message
    std::vector<const char *> bad(16, nullptr);
    host_parallel_chunks((size_t)m, nnz >= 1000000, [&](unsigned t, size_t i0, size_t i1) {
      for (size_t i = i0; i < i1; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
          const int32_t j = col_idx[k];
          const char *e = nullptr;
          if (j < 0 || j >= n) e = "column index out of range";
          else if (k > row_ptr[i] && col_idx[k - 1] >= j)
            e = "column indices not strictly increasing in a row";
          else if (!std::isfinite(val[k])) e = "non-finite matrix value";
          if (e) {
            bad[t] = e;
            return;
          }
        }
    });
    for (const char *e : bad)
      if (e) return fail(LP_ERR_INVALID, e);
  }
  for (int32_t j = 0; j < n; ++j) {
    if (!std::isfinite(c[j])) return fail(LP_ERR_INVALID, "non-finite cost");
    if (std::isnan(col_lo[j]) || std::isnan(col_hi[j]) || col_lo[j] > col_hi[j] ||
        col_lo[j] == INFINITY || col_hi[j] == -INFINITY)
      return fail(LP_ERR_INVALID, "invalid column bounds");
  }
  for (int32_t i = 0; i < m; ++i) {
    if (std::isnan(row_lo[i]) || std::isnan(row_hi[i]) || row_lo[i] > row_hi[i] ||
        row_lo[i] == INFINITY || row_hi[i] == -INFINITY)
      return fail(LP_ERR_INVALID, "invalid row bounds");
  }
  if (!std::isfinite(obj_offset)) return fail(LP_ERR_INVALID, "non-finite offset");
  // owned here until handed out: a failed copy (bad_alloc) releases it
  std::unique_ptr<lp_problem> lp(new lp_problem());
  HostLP &h = lp->cur;  // the original LP is the current one until presolve
  h.m = m;
  h.n = n;
  h.row_ptr.assign(row_ptr, row_ptr + m + 1);
  h.col_idx.assign(col_idx, col_idx + nnz);
  h.val.assign(val, val + nnz);
  h.c.assign(c, c + n);
  h.off = obj_offset;
  h.row_lo.assign(row_lo, row_lo + m);
  h.row_hi.assign(row_hi, row_hi + m);
  h.col_lo.assign(col_lo, col_lo + n);
  h.col_hi.assign(col_hi, col_hi + n);
  if (dev) {
    lp->has_dev = true;
    lp->dev = *dev;
  }
  *out = lp.release();
  return LP_OK;
  API_GUARD_END
}

int lp_presolve(lp_problem *lp, const lp_presolve_opts *opts, lp_presolve_info *info) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (lp->presolved) return fail(LP_ERR_STATE, "already presolved");
  lp_presolve_opts o;
  lp_presolve_opts_default(&o);
  if (opts) o = *opts;
  auto t0 = std::chrono::steady_clock::now();
  HostLP red;
  lp->orig = std::move(lp->cur);
  try {
    presolve_run(lp->orig, o.max_rounds, o.enable, red, lp->po);
  } catch (...) {
    lp->cur = std::move(lp->orig);
    lp->orig = HostLP();
    throw;
  }
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  lp->cur = std::move(red);
  lp->presolved = true;
  lp->sol = DeviceSolution();
  if (lp->dlp) {
    dev_destroy(lp->dlp);
    lp->dlp = nullptr;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = lp->po.status;
    info->rounds = lp->po.rounds;
    info->m = lp->cur.m;
    info->n = lp->cur.n;
    info->nnz = lp->cur.nnz();
    info->m0 = lp->orig.m;
    info->n0 = lp->orig.n;
    info->nnz0 = lp->orig.nnz();
    for (int q = 0; q < 16; ++q) info->counts[q] = lp->po.counts[q];
    info->seconds = secs;
  }
  return LP_OK;
  API_GUARD_END
}

int lp_upload(lp_problem *lp) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (!lp->has_dev) return fail(LP_ERR_STATE, "problem created without a device context");
  std::string err;
  if (!lp->dlp) {
    lp->dlp = dev_create(&lp->dev, err);
    if (!lp->dlp) return fail(LP_ERR_CUDA, err);
  }
  int rc = dev_upload(lp->dlp, lp->cur, err);
  if (rc != LP_OK) return fail(rc, err);
  return LP_OK;
  API_GUARD_END
}

int lp_solve(lp_problem *lp, const lp_solve_opts *opts, lp_result *res) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (!lp->has_dev) return fail(LP_ERR_STATE, "problem created without a device context");
  if (lp->presolved && lp->po.status != LP_PRESOLVE_REDUCED &&
      lp->po.status != LP_PRESOLVE_SOLVED) {
    if (res) {
      std::memset(res, 0, sizeof(*res));
      res->termination = lp->po.status == LP_PRESOLVE_INFEASIBLE ? LP_INFEASIBLE : LP_UNBOUNDED;
    }
    return LP_OK;
  }
  lp_solve_opts o;
  lp_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_solve_opts(o)) return fail(LP_ERR_INVALID, "invalid solve options");
  std::string err;
  auto solve_once = [&](const lp_solve_opts &oo, lp_result &r) -> int {
    std::memset(&r, 0, sizeof(r));
    const bool cluster = oo.engine == LP_ENGINE_CLUSTER ||
                         (oo.engine == LP_ENGINE_AUTO && !oo.polish &&
                          lp->cur.nnz() < kClusterEngineNnz);
    if (cluster) return cluster_solve(lp->cur, oo, &lp->dev, &r, lp->sol, err);
    if (!lp->dlp) {
      lp->dlp = dev_create(&lp->dev, err);
      if (!lp->dlp) return LP_ERR_CUDA;
    }
    if (!dev_uploaded(lp->dlp)) {
      int rc = dev_upload(lp->dlp, lp->cur, err);
      if (rc != LP_OK) return rc;
    }
    return dev_solve(lp->dlp, lp->cur, oo, &r, lp->sol, err);
  };
  const auto t0 = std::chrono::steady_clock::now();
  lp_result r;
  int rc = solve_once(o, r);
  if (rc != LP_OK) return fail(rc, err);
  r.rel_kkt_original = r.rel_kkt;
  r.refinements = 0;
  // postsolve amplification: the reduced LP's rel-KKT bounds the original
  // LP's only up to the postsolve's conditioning; while the postsolved point
  // misses eps_rel on the original LP, solve the reduced LP again ten times
  // tighter, warm-started from the last solution
  if (lp->presolved && o.refine_original > 0 && r.termination == LP_OPTIMAL) {
    double eps = o.eps_rel;
    for (int q = 0;; ++q) {
      double kk[9];
      problem_original_measures(lp, lp->sol.x.data(), lp->sol.y.data(), lp->sol.z.data(), kk);
      r.rel_kkt_original = kk[0];
      // the stopping test on the original LP (rel_p, rel_d, rel_gap)
      const double eg = o.eps_gap_rel > 0 ? o.eps_gap_rel : o.eps_rel;
      const bool met = kk[1] <= o.eps_rel && kk[2] <= o.eps_rel && kk[3] <= eg;
      if (met || q == o.refine_original || r.termination != LP_OPTIMAL) break;
      eps *= 0.1;
      const std::vector<double> xw = lp->sol.x, yw = lp->sol.y;
      lp_solve_opts o2 = o;
      o2.eps_rel = eps;
      if (o.eps_gap_rel > 0) o2.eps_gap_rel = o.eps_gap_rel * std::pow(0.1, q + 1);
      o2.x_init = xw.data();
      o2.y_init = yw.data();
      lp_result r2;
      rc = solve_once(o2, r2);
      if (rc != LP_OK) return fail(rc, err);
      r2.iterations += r.iterations;
      r2.restarts += r.restarts;
      r2.t_setup_s += r.t_setup_s;
      r2.t_solve_s += r.t_solve_s;
      r2.kernel_launches += r.kernel_launches;
      r2.fp32_iterations += r.fp32_iterations;
      r2.refinements = r.refinements + 1;
      r = r2;
    }
    r.t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  lp->last_termination = r.termination;
  if (res) *res = r;
  return LP_OK;
  API_GUARD_END
}

int lp_get_solution(const lp_problem *lp, double *x, double *y, double *z) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (!lp->sol.valid) return fail(LP_ERR_STATE, "no solution yet");
  if (x) std::memcpy(x, lp->sol.x.data(), sizeof(double) * lp->cur.n);
  if (y) std::memcpy(y, lp->sol.y.data(), sizeof(double) * lp->cur.m);
  if (z) std::memcpy(z, lp->sol.z.data(), sizeof(double) * lp->cur.n);
  return LP_OK;
  API_GUARD_END
}

int lp_get_iterate(const lp_problem *lp, double *x, double *y) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (!lp->sol.valid) return fail(LP_ERR_STATE, "no solution yet");
  if (x) std::memcpy(x, lp->sol.xi.data(), sizeof(double) * lp->cur.n);
  if (y) std::memcpy(y, lp->sol.yi.data(), sizeof(double) * lp->cur.m);
  return LP_OK;
  API_GUARD_END
}

int lp_postsolve_from(lp_problem *lp, const double *xr, const double *yr, const double *zr,
                      double *x, double *y, double *z) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if ((lp->cur.n && !xr) || (lp->cur.m && !yr)) return fail(LP_ERR_INVALID, "NULL input");
  const HostLP &orig = original_lp(lp);
  std::vector<double> X(orig.n), Y(orig.m), Z(orig.n);
  if (!lp->presolved) {
    std::copy(xr, xr + lp->cur.n, X.begin());
    std::copy(yr, yr + lp->cur.m, Y.begin());
    if (zr) {
      std::copy(zr, zr + lp->cur.n, Z.begin());
    } else {
      const HostLP &h = lp->cur;
      Z = h.c;
      for (int32_t i = 0; i < h.m; ++i)
        for (int64_t k = h.row_ptr[i]; k < h.row_ptr[i + 1]; ++k)
          Z[h.col_idx[k]] -= h.val[k] * yr[i];
    }
  } else {
    postsolve_run(lp->po, lp->cur, xr, yr, zr, X.data(), Y.data(), Z.data());
  }
  if (x) std::memcpy(x, X.data(), sizeof(double) * X.size());
  if (y) std::memcpy(y, Y.data(), sizeof(double) * Y.size());
  if (z) std::memcpy(z, Z.data(), sizeof(double) * Z.size());
  return LP_OK;
  API_GUARD_END
}

int lp_postsolve(lp_problem *lp, double *x, double *y, double *z) {
  API_GUARD_BEGIN
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (!lp->sol.valid) {
    if (lp->cur.m == 0 && lp->cur.n == 0) {
      // presolve removed everything: postsolve from the empty solution
      return lp_postsolve_from(lp, nullptr, nullptr, nullptr, x, y, z);
    }
    return fail(LP_ERR_STATE, "no solution to postsolve");
  }
  return lp_postsolve_from(lp, lp->sol.x.data(), lp->sol.y.data(), lp->sol.z.data(), x, y, z);
  API_GUARD_END
}

int lp_get_dims(const lp_problem *lp, int32_t *m, int32_t *n, int64_t *nnz, int32_t *m0,
                int32_t *n0) {
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  if (m) *m = lp->cur.m;
  if (n) *n = lp->cur.n;
  if (nnz) *nnz = lp->cur.nnz();
  if (m0) *m0 = original_lp(lp).m;
  if (n0) *n0 = original_lp(lp).n;
  return LP_OK;
}

int lp_get_data(const lp_problem *lp, int64_t *row_ptr, int32_t *col_idx, double *val,
                double *c, double *obj_offset, double *row_lo, double *row_hi,
                double *col_lo, double *col_hi) {
  if (!lp) return fail(LP_ERR_INVALID, "lp is NULL");
  const HostLP &h = lp->cur;
  if (row_ptr) std::memcpy(row_ptr, h.row_ptr.data(), sizeof(int64_t) * (h.m + 1));
  if (col_idx && h.nnz()) std::memcpy(col_idx, h.col_idx.data(), sizeof(int32_t) * h.nnz());
  if (val && h.nnz()) std::memcpy(val, h.val.data(), sizeof(double) * h.nnz());
  if (c && h.n) std::memcpy(c, h.c.data(), sizeof(double) * h.n);
  if (obj_offset) *obj_offset = h.off;
  if (row_lo && h.m) std::memcpy(row_lo, h.row_lo.data(), sizeof(double) * h.m);
  if (row_hi && h.m) std::memcpy(row_hi, h.row_hi.data(), sizeof(double) * h.m);
  if (col_lo && h.n) std::memcpy(col_lo, h.col_lo.data(), sizeof(double) * h.n);
  if (col_hi && h.n) std::memcpy(col_hi, h.col_hi.data(), sizeof(double) * h.n);
  return LP_OK;
}

int lp_host_rel_kkt(const lp_problem *lp, const double *x, const double *y, double *out) {
  API_GUARD_BEGIN
  if (!lp || !out) return fail(LP_ERR_INVALID, "NULL argument");
  double o[9];
  host_rel_kkt(lp->cur, x, y, o);
  for (int q = 0; q < 6; ++q) out[q] = o[q];
  return LP_OK;
  API_GUARD_END
}

int lp_profile_kernels(lp_problem *lp, int32_t reps, double *out) {
  API_GUARD_BEGIN
  if (!lp || !out || reps < 1) return fail(LP_ERR_INVALID, "invalid argument");
  if (!lp->dlp) return fail(LP_ERR_STATE, "profile needs a prior solve");
  std::string err;
  int rc = dev_profile(lp->dlp, reps, out, err);
  if (rc != LP_OK) return fail(rc, err);
  return LP_OK;
  API_GUARD_END
}

int lp_get_tile_tuning(const lp_problem *lp, double *out, int32_t cap, int32_t *count) {
  API_GUARD_BEGIN
  if (!lp || !out || !count) return fail(LP_ERR_INVALID, "NULL argument");
  if (!lp->dlp || !dev_uploaded(lp->dlp))
    return fail(LP_ERR_STATE, "no grid-engine solve on this problem");
  const int k = dev_tile_tuning(lp->dlp, out, cap);
  if (k < 0) return fail(LP_ERR_INVALID, "cap too small");
  *count = k;
  return LP_OK;
  API_GUARD_END
}

void lp_tile_cache_clear(void) {
  dev_tile_cache_clear();
  batch_tile_cache_clear();
}

void lp_destroy(lp_problem *lp) {
  if (!lp) return;
  try {
    if (lp->dlp) dev_destroy(lp->dlp);
  } catch (...) {
  }
  delete lp;
}

}  // extern "C"

namespace gb300lp {

// rel-KKT (the termination measure): r_p = ||Ax - proj(Ax)||, lam =
// proj_Lambda(c - A^T y) with the sign sets of eq. (2), r_d = ||(c - A^T y -
// lam, y - proj_Y(y))||, p = c^T x + off, d = support terms + off,
// rel = max(r_p / (1 + ||bhat||), r_d / (1 + ||c||), |p - d| / (1 + |p| + |d|)).
void host_rel_kkt(const HostLP &h, const double *x, const double *y, double out[9]) {
  std::vector<double> g(h.c);
  double rp2 = 0, rd2 = 0, dsum = 0, bn2 = 0, cn2 = 0, p = h.off;
  for (int32_t i = 0; i < h.m; ++i) {
    double ax = 0;
    for (int64_t k = h.row_ptr[i]; k < h.row_ptr[i + 1]; ++k) {
      ax += h.val[k] * x[h.col_idx[k]];
      g[h.col_idx[k]] -= h.val[k] * y[i];
    }
    double lo = h.row_lo[i], hi = h.row_hi[i];
    double pr = std::fmin(std::fmax(ax, lo), hi);
    rp2 += (ax - pr) * (ax - pr);
    double yp = y[i];
    if (!std::isfinite(lo)) yp = std::fmin(yp, 0.0);
    if (!std::isfinite(hi)) yp = std::fmax(yp, 0.0);
    rd2 += (y[i] - yp) * (y[i] - yp);
    if (yp > 0) dsum += yp * lo;
    else if (yp < 0) dsum += yp * hi;
    if (std::isfinite(lo)) bn2 += lo * lo;
    if (std::isfinite(hi) && !(std::isfinite(lo) && lo == hi)) bn2 += hi * hi;
  }
  for (int32_t j = 0; j < h.n; ++j) {
    double lf = std::isfinite(h.col_lo[j]), uf = std::isfinite(h.col_hi[j]);
    double lam = g[j];
    if (!lf && !uf) lam = 0;
    else if (lf && !uf) lam = std::fmax(lam, 0.0);
    else if (!lf && uf) lam = std::fmin(lam, 0.0);
    rd2 += (g[j] - lam) * (g[j] - lam);
    if (lam > 0) dsum += lam * h.col_lo[j];
    else if (lam < 0) dsum += lam * h.col_hi[j];
    p += h.c[j] * x[j];
    cn2 += h.c[j] * h.c[j];
  }
  double d = dsum + h.off;
  double rp = std::sqrt(rp2), rd = std::sqrt(rd2), gap = std::fabs(p - d);
  double relp = rp / (1 + std::sqrt(bn2)), reld = rd / (1 + std::sqrt(cn2));
  double relg = gap / (1 + std::fabs(p) + std::fabs(d));
  out[0] = std::fmax(relp, std::fmax(reld, relg));
  out[1] = relp;
  out[2] = reld;
  out[3] = relg;
  out[4] = p;
  out[5] = d;
  out[6] = rp;
  out[7] = rd;
  out[8] = gap;
}

}  // namespace gb300lp
