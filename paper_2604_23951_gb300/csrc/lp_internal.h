// Internal C++ interfaces shared by the host (api, presolve) and device
// (solver, batch) translation units.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "lp.h"

namespace gb300lp {

// CSR problem of eq. (1) held on the host.
struct HostLP {
  int32_t m = 0, n = 0;
  std::vector<int64_t> row_ptr{0};
  std::vector<int32_t> col_idx;
  std::vector<double> val;
  std::vector<double> c;
  double off = 0.0;
  std::vector<double> row_lo, row_hi, col_lo, col_hi;
  int64_t nnz() const { return row_ptr.empty() ? 0 : row_ptr.back(); }
};

// Relative KKT error of (x, y) for `lp` (the measure of the termination test,
// written on the host in FP64).  out: rel_kkt, rel_p, rel_d, rel_gap, p, d,
// r_p, r_d, gap.
void host_rel_kkt(const HostLP &lp, const double *x, const double *y, double out[9]);

// lp_solve_opts within their documented ranges (api.cpp)
bool valid_solve_opts(const lp_solve_opts &o);

// ---- presolve (presolve.cpp) -------------------------------------------
struct PostsolveRecord {
  int32_t kind;  // see presolve.cpp
  int32_t i, j, k;
  double a, b, cj, v, ak;
  int32_t flags;             // bit 0: lower bound came from the row / column
                             // bit 1: upper bound came from the row / column
  int64_t ent_begin, ent_end;  // slice of the entry pool
};

struct PresolveOutcome {
  int32_t status = LP_PRESOLVE_REDUCED;
  int32_t rounds = 0;
  int64_t counts[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<PostsolveRecord> records;
  std::vector<int32_t> ent_idx;
  std::vector<double> ent_val;
  std::vector<int32_t> row_map, col_map;  // reduced -> original
  int32_t m0 = 0, n0 = 0;
};

// Presolve `in` (the original LP); on success `out` is the reduced LP.
void presolve_run(const HostLP &in, int max_rounds, int rule_mask, HostLP &out,
                  PresolveOutcome &po);

// Replay the postsolve records (reverse order) from a reduced solution.
void postsolve_run(const PresolveOutcome &po, const HostLP &reduced, const double *xr,
                   const double *yr, const double *zr, double *x, double *y, double *z);

// ---- device single-LP path (solver.cu) -----------------------------------
struct DeviceLP;

struct DeviceSolution {
  std::vector<double> x, y, z;   // T(z) at termination (unscaled, original order)
  std::vector<double> xi, yi;    // iterate z^t
  bool valid = false;
};

DeviceLP *dev_create(const lp_device_ctx *ctx, std::string &err);
int dev_upload(DeviceLP *d, const HostLP &lp, std::string &err);
bool dev_uploaded(const DeviceLP *d);
int dev_solve(DeviceLP *d, const HostLP &lp, const lp_solve_opts &opts, lp_result *res,
              DeviceSolution &sol, std::string &err);
void dev_destroy(DeviceLP *d);
int dev_profile(DeviceLP *d, int reps, double *out, std::string &err);
// the grid engine's tile-shape autotuner: forget every cached choice; report
// the last solve's shapes and measurement (lp_get_tile_tuning's layout;
// -1 if cap is too small)
void dev_tile_cache_clear();
// the batched path's tile-shape classes (batch.cu)
void batch_tile_cache_clear();
int dev_tile_tuning(const DeviceLP *d, double *out, int cap);

// Per-check trace: when the environment variable LP_TRACE names a file, one
// JSON line per state read-back of a solve is appended to it (api.cpp).
void trace_state(const char *engine, long long t, double rel_kkt, double rel_p, double rel_d,
                 double rel_gap, double omega, int restarts, int fp32);

// The cluster engine: one thread-block cluster runs the whole solve of a
// small LP (batch.cu); same algorithm and result semantics as dev_solve.
int cluster_solve(const HostLP &lp, const lp_solve_opts &opts, const lp_device_ctx *ctx,
                  lp_result *res, DeviceSolution &sol, std::string &err);
constexpr long long kClusterEngineNnz = 4096;  // LP_ENGINE_AUTO picks it below this size

// ---- shared device-memory helpers (solver.cu) ----------------------------
struct DevAlloc {
  lp_device_ctx ctx{};
  bool own_stream = false;
  void *stream = nullptr;
  int device = 0;
};

}  // namespace gb300lp
