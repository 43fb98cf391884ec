/*
 * lp.h -- C ABI of the GB300 restarted-PDHG LP library.
 *
 * Problem (eq. (1), Sec. 2):   minimize  c^T x + obj_offset
 *                              subject to row_lo <= A x <= row_hi
 *                                         col_lo <= x  <= col_hi
 * A is m x n, given in CSR.  Infinite bounds are IEEE +-INFINITY; an equality
 * row has row_lo[i] == row_hi[i].  A solution is (x, y, z) satisfying the
 * optimality conditions of eq. (2): primal feasibility, c - A^T y - z = 0 and
 * the sign / complementarity rules for y and z.
 *
 * Pipeline (Sec. 1, Sec. 3.3): lp_create -> lp_presolve (host, the simple
 * rules of Sec. 2-3, keeps a postsolve record) -> lp_solve (GPU restarted
 * reflected Halpern PDHG on the reduced LP) -> lp_postsolve (host, maps the
 * reduced solution back to an (x, y, z) of the original LP).  The presolve
 * interface follows the minimal pointer-in / same-form-out design of Sec. 3.3.
 *
 * Conventions shared by every entry point:
 *   - All pointers passed in are HOST pointers unless stated otherwise.  Input
 *     arrays are copied; the caller keeps ownership and may free them once
 *     the call returns.  Output arrays are caller-allocated host buffers.
 *   - Return codes: LP_OK (0) on success, LP_PENDING (1) from lp_batch_poll
 *     while a request is in flight, a negative LP_ERR_* code on failure.
 *     lp_last_error() returns a message for the last failure on the calling
 *     thread.  No C++ exception and no abort crosses this boundary.
 *   - Device work runs on the CUDA stream given in lp_device_ctx (NULL = the
 *     library creates its own non-blocking stream).  Device memory comes from
 *     the ctx allocator callbacks when given, else from cudaMallocAsync.
 *   - Sizes: m, n < 2^31; nnz < 2^31 on the device (checked at upload).
 */
#ifndef GB300_LP_H
#define GB300_LP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define LP_OK 0
#define LP_PENDING 1
#define LP_ERR_INVALID (-1) /* malformed input (NaN, bad CSR, lo > hi, ...)   */
#define LP_ERR_OOM (-2)     /* host or device allocation failed              */
#define LP_ERR_CUDA (-3)    /* a CUDA runtime call failed                    */
#define LP_ERR_STATE (-4)   /* call not valid in the object's current state  */
#define LP_ERR_BUDGET (-5)  /* request larger than the server's HBM budget   */
#define LP_ERR_TIMEOUT (-6) /* reserved: no call returns it (no device wait) */

/* ---- termination codes (lp_result.termination) ------------------------ */
#define LP_OPTIMAL 0    /* the stopping test holds: rel_p, rel_d <= eps_rel and
                         * rel_gap <= eps_gap_rel (default: rel-KKT <= eps_rel) */
#define LP_ITER_LIMIT 1 /* max_iter iterations done                          */
#define LP_TIME_LIMIT 2 /* time_limit_s elapsed                              */
#define LP_NUMERICAL 3  /* a non-finite value appeared                       */
#define LP_INFEASIBLE 4 /* presolve proved the LP infeasible, or the solver
                           found a dual ray (Farkas certificate)             */
#define LP_UNBOUNDED 5  /* presolve proved the LP unbounded, or the solver
                           found a primal ray (the dual is infeasible)       */
#define LP_CANCELLED 6  /* batch request cancelled                           */

/* ---- presolve status (lp_presolve_info.status) ------------------------- */
#define LP_PRESOLVE_REDUCED 0
#define LP_PRESOLVE_INFEASIBLE 1
#define LP_PRESOLVE_UNBOUNDED 2
#define LP_PRESOLVE_SOLVED 3 /* every row and column was removed            */

/* ---- engine (lp_solve_opts.engine) ------------------------------------- */
#define LP_ENGINE_AUTO 0
#define LP_ENGINE_GRID 1
#define LP_ENGINE_CLUSTER 2

/* ---- precision (lp_solve_opts.precision) ------------------------------- */
#define LP_FP64 0  /* FP64 matrix, FP64 SpMV, FP64 everything               */
#define LP_MIXED 1 /* FP32 matrix values times vectors gathered as float    */
                   /* pairs, compensated FP32 sums; iterates, anchor,        */
                   /* reductions, restarts stay FP64 (see lp_solve)          */

typedef struct lp_problem lp_problem; /* opaque: host copy + device buffers */
typedef struct lp_server lp_server;   /* opaque: continuous-batching server  */

/* Device context.  alloc(bytes, user) returns device memory or NULL; free
 * releases it.  Both NULL: the library uses cudaMallocAsync / cudaFreeAsync
 * on `stream`.  `stream` is a cudaStream_t (NULL: the library creates one).
 * The callbacks are only invoked from the thread that calls into the library
 * (a server calls alloc once, at lp_server_create). */
typedef struct {
  void *(*alloc)(size_t bytes, void *user);
  void (*free)(void *ptr, void *user);
  void *user;
  void *stream;
  int32_t device;
} lp_device_ctx;

typedef struct {
  int32_t max_rounds; /* 20: stop after this many rounds                     */
  int32_t enable;     /* bit mask of rules, LP_RULE_ALL by default           */
} lp_presolve_opts;

#define LP_RULE_EMPTY_ROW 1
#define LP_RULE_EMPTY_COL 2
#define LP_RULE_FIXED_COL 4
#define LP_RULE_SINGLETON_ROW 8
#define LP_RULE_REDUNDANT_ROW 16
#define LP_RULE_DOUBLETON 32
#define LP_RULE_FREE_COL_SINGLETON 64
#define LP_RULE_VARIABLE_LOCKS 128 /* weak dual fixing (Sec. 2.3)             */
#define LP_RULE_COL_SINGLETON_INEQ 256 /* column singleton in an inequality
                                          row: the row becomes an equality
                                          at the side every optimum is at  */
#define LP_RULE_PARALLEL_ROWS 512  /* medium explorer (Table 1): run when a
                                      round of the others changed nothing  */
#define LP_RULE_ALL 1023
#define LP_RULE_DUAL_PROPAGATION 4096 /* medium explorer (Table 1), not in
                                         LP_RULE_ALL: one sweep of dual
                                         bounds from the columns' dual
                                         constraints; rows with a signed dual
                                         become equalities, columns with a
                                         signed reduced cost are fixed       */
#define LP_RULE_PARALLEL_COLS 2048 /* medium explorer (Table 1), not in
                                      LP_RULE_ALL: columns with a_k = s a_j
                                      and c_k = s c_j become one variable
                                      x_j + s x_k (split again in postsolve) */
#define LP_RULE_PRIMAL_PROPAGATION 1024 /* medium explorer (Table 1), not in
                                           LP_RULE_ALL: bounds implied by the
                                           rows' activities (a tightened bound
                                           that ends active hands its reduced
                                           cost to the row in postsolve)     */

typedef struct {
  int32_t status;          /* LP_PRESOLVE_*                                 */
  int32_t rounds;
  int32_t m, n;            /* reduced sizes                                 */
  int64_t nnz;
  int32_t m0, n0;          /* original sizes                                */
  int64_t nnz0;
  int64_t counts[16];      /* reductions per rule: empty_row, empty_col,
                              fixed_col, singleton_row, redundant_row,
                              dropped_side, doubleton, free_col_singleton,
                              variable locks (dual fixing), inequality
                              rows made equalities, parallel rows merged,
                              bounds tightened by primal propagation,
                              parallel columns merged, dual propagation
                              (rows made equalities + columns fixed);
                              14-15 unused                                 */
  double seconds;
} lp_presolve_info;

typedef struct {
  double eps_rel;        /* 1e-6: stop when relative KKT error <= eps_rel   */
  int64_t max_iter;      /* 200000                                          */
  double time_limit_s;   /* 3600                                            */
  int32_t precision;     /* LP_FP64 | LP_MIXED                              */
  int32_t check_every;   /* 64: restart/termination check period K          */
  double rho;            /* 1.0: reflection weight (0 = plain Halpern)      */
  double beta_suff;      /* 0.2  restart if r <= beta_suff r0               */
  double beta_nec;       /* 0.8  ... or r <= beta_nec r0 and r > r_prev     */
  double beta_art;       /* 0.36 ... or k >= beta_art t                     */
  double theta;          /* 0.5  primal-weight smoothing                    */
  int32_t ruiz_iters;    /* 10                                              */
  int32_t pock_chambolle;/* 1                                               */
  int32_t power_iters;   /* 100                                             */
  int32_t halpern;       /* 1: Halpern anchoring; 0: (1+rho)T(z) - rho z    */
  int32_t restarts;      /* 1: restarts enabled                             */
  int32_t use_graph;     /* 1: replay a CUDA graph of check_every iterations
                          * (grid engine); the server replays one graph per
                          * bucket launch (lp_server_graph_stats)           */
  double step_size;      /* 0 = auto: 0.998 / ||A~||_2 by power iteration   */
  double primal_weight;  /* 0 = auto: ||c~|| / ||bhat~||                    */
  const double *x_init;  /* NULL or n doubles (current LP): warm start x    */
  const double *y_init;  /* NULL or m doubles: warm start y                 */
  int32_t engine;        /* LP_ENGINE_AUTO (0): the cluster engine for LPs
                          * under 4,096 nonzeros, the grid engine
                          * otherwise; LP_ENGINE_GRID (1): CUDA-graph
                          * replay of the grid-wide kernels;
                          * LP_ENGINE_CLUSTER (2): one thread-block cluster
                          * (1-8 CTAs by size) runs the whole solve.  Both
                          * run the same algorithm with the same results
                          * semantics; use_graph and lp_profile_kernels
                          * concern the grid engine only.                  */
  int32_t verbose;
  int32_t infeas_every;  /* 4: at every infeas_every-th check the direction
                          * d = T(z) - z0 since the last restart is tested
                          * for a certificate (0: never).  Dual ray: w =
                          * d_y projected on the rows' sign domain, lam =
                          * proj_Lambda(-A^T w), dual objective D =
                          * sum(w+ l_c - w- u_c) + sum(lam+ l_x - lam- u_x);
                          * LP_INFEASIBLE when D > 0 and ||A^T w + lam||_2
                          * <= eps_infeas D.  Primal ray: d_x with c^T d_x
                          * < 0 whose violation of the recession cones of
                          * [l_c, u_c] (for A d_x) and [l_x, u_x] is at most
                          * eps_infeas (-c^T d_x) in 2-norm: LP_UNBOUNDED.
                          * All in the LP's own units; the returned x, y
                          * are T(z) of that check.                         */
  double eps_infeas;     /* 1e-8                                            */
  double primal_weight_clamp; /* 10: after each primal-weight update omega
                          * stays within [omega_0 / c, omega_0 * c], omega_0
                          * the initial weight (0: no bound; else >= 1)     */
  int32_t refine_original; /* 3: for a presolved problem, after an optimal
                          * solve the reduced solution is postsolved and its
                          * rel-KKT measured on the ORIGINAL LP (host, FP64);
                          * while that exceeds eps_rel (postsolve can amplify
                          * the reduced LP's error), the reduced LP is solved
                          * again with a tolerance ten times tighter, warm-
                          * started from the last solution, at most this many
                          * times (0: no check).  Applies to lp_solve and to
                          * served requests (lp_batch_poll).                 */
  int32_t tile_run_max;  /* grid engine tile shape: most entries one lane
                          * owns in a row (8, 16, 32 or 64) ...             */
  int32_t tile_nnz;      /* ... and nonzeros per warp tile (512 or 2048);
                          * either 0 (default): the autotuner's choice for
                          * each matrix (A and A^T separately), measured on
                          * the first solve of a size class and kept for the
                          * process.  Results are bitwise reproducible for a
                          * fixed shape; different shapes sum in a different
                          * order.                                          */
  double eps_gap_rel;    /* 0 (= eps_rel): the stopping test is rel_p <=
                          * eps_rel, rel_d <= eps_rel and rel_gap <= this
                          * (with 0 exactly relative KKT error <= eps_rel)  */
  int32_t polish;        /* 0; 1: feasibility polishing (grid engine only;
                          * LP_ENGINE_AUTO then picks the grid engine).  At
                          * a check at t >= the next allowed attempt where
                          * rel_gap <= eps_gap_rel but rel_p or rel_d >
                          * eps_rel, two PDHG phases start from that check's
                          * T(z) = (x^, y^): the LP with c = 0 from (x^, 0)
                          * until rel_p <= eps_rel, then the LP with every
                          * finite bound set to 0 from (0, y^) until rel_d <=
                          * eps_rel (the original LP's rel_p / rel_d), each
                          * a fresh restarted Halpern PDHG with the solve's
                          * step size and omega_0 = the current weight, no
                          * infeasibility test, at most max(K, polish_fraction
                          * t) iterations rounded up to a multiple of K.
                          * If both succeed and their pair (x, y) meets the
                          * stopping test on the original LP, it is returned
                          * (LP_OPTIMAL); otherwise the solve resumes at that
                          * check and the next attempt waits until 2 t.
                          * Meant for eps_gap_rel well above eps_rel: the
                          * phases move the objective values.  The phases'
                          * iterations count in lp_result.iterations.       */
  int32_t pad_polish_;
  double polish_fraction; /* 0.125 (0 < f <= 8)                             */
} lp_solve_opts;

typedef struct {
  int32_t termination;   /* LP_OPTIMAL ...                                   */
  int32_t restarts;
  int64_t iterations;    /* evaluations of the PDHG operator T              */
  double rel_kkt, rel_p, rel_d, rel_gap;
  double r_p, r_d, gap;
  double primal_obj, dual_obj;
  double eta, omega;
  double t_setup_s;      /* scaling + step size (device)                    */
  double t_solve_s;      /* PDHG iterations (device)                        */
  double t_total_s;      /* wall time of the call                           */
  int64_t kernel_launches; /* kernels launched by this call                 */
  int64_t fp32_iterations; /* LP_MIXED: iterations run with the FP32 SpMV
                              before the switch to FP64 (see lp_solve)      */
  double rel_kkt_original; /* rel-KKT of the postsolved point on the original
                              LP (host, FP64) when the problem was presolved
                              and refine_original > 0; otherwise the same as
                              rel_kkt (the current LP is the original)      */
  int32_t refinements;     /* re-solves at a tighter tolerance that the
                              original-LP check asked for (iterations and
                              times above include them)                     */
  int32_t polish_attempts; /* feasibility-polishing attempts (opts.polish)  */
  int32_t polished;        /* 1: the returned point is a polished pair      */
  int32_t pad_;
  int64_t polish_iterations; /* iterations of the polishing phases         */
} lp_result;

/* Defaults above; always call before filling in a field. */
void lp_solve_opts_default(lp_solve_opts *opts);
void lp_presolve_opts_default(lp_presolve_opts *opts);

/* Thread-local message for the last failing call on this thread. */
const char *lp_last_error(void);

/* Create a problem from CSR (row_ptr: m+1 int64, col_idx: nnz int32 strictly
 * increasing within each row, val: nnz doubles), c (n), bounds.  dev may be
 * NULL (host-only: presolve/postsolve work, lp_solve fails LP_ERR_STATE).
 * Fails LP_ERR_INVALID on NaN, a decreasing row_ptr, an out-of-range or
 * repeated column index in a row, lo > hi, +inf lower or -inf upper bound. */
int lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
              const int32_t *col_idx, const double *val, const double *c,
              double obj_offset, const double *row_lo, const double *row_hi,
              const double *col_lo, const double *col_hi,
              const lp_device_ctx *dev, lp_problem **out);

/* Presolve in place (Sec. 2-3): the problem becomes the reduced LP; the
 * postsolve record is kept inside.  Host only.  May be called once.  Each
 * round runs the enabled passes in the order empty rows, empty columns,
 * fixed columns, singleton rows, redundant rows / dominated row sides,
 * doubleton equalities, column singletons in inequality rows, free column
 * singletons, variable locks; round 1 scans everything, later rounds what
 * the previous round changed.  A round in which these change nothing runs
 * the medium explorers over every row / column: primal propagation (if
 * enabled), dual propagation (if enabled, once), parallel rows, parallel
 * columns (if enabled); the rounds end
 * when they find nothing either (or after max_rounds).  Parts run on several host threads;
 * the result does not depend on the thread count. */
int lp_presolve(lp_problem *lp, const lp_presolve_opts *opts, lp_presolve_info *info);

/* Copy the current (reduced) LP to the device and build its layout (row
 * binning and the stored transpose).  lp_solve calls it when needed. */
int lp_upload(lp_problem *lp);

/* Solve the current (reduced) LP on the GPU.  May be called repeatedly;
 * every call starts from the initial (or warm-start) point.  LP_MIXED runs
 * the SpMV on FP32 matrix values (the gathered vectors as float pairs,
 * compensated FP32 sums; everything else FP64) and switches to the FP64
 * SpMV for good only if the best relative KKT error has not halved over 256
 * checks; the iterates, anchor and weights carry over.  When the
 * environment variable LP_TRACE names a file, every state read-back (each
 * check period of the grid engine, each launch of the cluster engine)
 * appends one JSON line: engine, t, rel_kkt, rel_p, rel_d, rel_gap, omega,
 * restarts, fp32. */
int lp_solve(lp_problem *lp, const lp_solve_opts *opts, lp_result *res);

/* Solution of the current (reduced) LP: x (n), y (m), z = c - A^T y (n).
 * Any pointer may be NULL. */
int lp_get_solution(const lp_problem *lp, double *x, double *y, double *z);

/* The PDHG iterate z^t = (x, y) after the last lp_solve (unscaled). */
int lp_get_iterate(const lp_problem *lp, double *x, double *y);

/* Map the reduced solution back to the original LP (Sec. 2.1, Sec. 3.3):
 * x (n0), y (m0), z (n0), any may be NULL.  Without a presolve it copies. */
int lp_postsolve(lp_problem *lp, double *x, double *y, double *z);

/* Postsolve an externally supplied reduced solution (xr: n, yr: m, zr: n or
 * NULL for c - A^T yr) into original-size x, y, z. */
int lp_postsolve_from(lp_problem *lp, const double *xr, const double *yr,
                      const double *zr, double *x, double *y, double *z);

/* Current LP data (after presolve: the reduced LP).  Arrays may be NULL. */
int lp_get_dims(const lp_problem *lp, int32_t *m, int32_t *n, int64_t *nnz,
                int32_t *m0, int32_t *n0);
int lp_get_data(const lp_problem *lp, int64_t *row_ptr, int32_t *col_idx,
                double *val, double *c, double *obj_offset, double *row_lo,
                double *row_hi, double *col_lo, double *col_hi);

/* Relative KKT error (rel-KKT of the termination test) of a host point (x,
 * y) for the current LP, computed on the host in FP64. out: rel_kkt, rel_p,
 * rel_d, rel_gap, primal_obj, dual_obj (6 doubles). */
int lp_host_rel_kkt(const lp_problem *lp, const double *x, const double *y, double *out);

/* The row plan of the device layout, for `rows` rows of lengths len[]:
 * perm[new] = old row (longest first; equal lengths in their original
 * order -- the same order for every tile shape);
 * *nlong = the number of rows longer than 512 (each reduced by one CTA);
 * tiles[2 t], tiles[2 t + 1] = first row and packed word (nrows | lanes_log2
 * << 8 | entries_per_lane << 12) of warp tile t, for t < *ntiles.  tiles
 * holds `tile_cap` pairs; LP_ERR_INVALID (and *ntiles = the count needed) if
 * that is too few.  Host only; no device needed. */
int lp_plan_rows(int32_t rows, const int64_t *len, int32_t *perm, int32_t *tiles,
                 int32_t tile_cap, int32_t *ntiles, int32_t *nlong);

/* The same under a given tile shape: run_max (1..64) most entries a lane owns
 * in a row (2^v lanes per row, v the least with 2^v * run_max >= the tile's
 * longest row L; a lane walks its share in c = ceil(L / (2^v * 8)) chunks of
 * nit = ceil(L / (2^v c)) entries), tile_nnz (>= 32) nonzeros a tile aims at
 * (min(32, tile_nnz / L) rows).  segmented != 0: rows longer than
 * 32 * run_max come first and are cut into segments of 32 * run_max entries,
 * one tile each: tiles[2 t] = the row, tiles[2 t + 1] = INT_MIN | segment
 * index, and seg_base (seg_cap ints, may be NULL) receives *nsegrows + 1
 * offsets: row r's segments are seg_base[r] .. seg_base[r + 1] - 1; *nlong is
 * then 0.  segmented == 0: rows longer than 512 are CTA rows (*nlong) and
 * rows in (32 * run_max, 512] single-row tiles, as lp_plan_rows (which is
 * run_max 8, tile_nnz 512, unsegmented). */
int lp_plan_rows_shape(int32_t rows, const int64_t *len, int32_t run_max, int32_t tile_nnz,
                       int32_t segmented, int32_t *perm, int32_t *tiles, int32_t tile_cap,
                       int32_t *ntiles, int32_t *nlong, int32_t *seg_base, int32_t seg_cap,
                       int32_t *nsegrows);

/* Measurement hook (no counterpart in the paper): time the PDHG iteration
 * kernels of the last lp_solve one launch at a time with CUDA events on the
 * problem's stream, each launch after a 256 MiB write that evicts L2.
 * reps >= 1.  out (8 doubles): mean ms of the primal kernel (A^T y + primal
 * epilogue), mean ms of the dual kernel (A xbar + dual epilogue), their
 * algorithmic bytes per launch, then the same four for the two KKT kernels.
 * Fails LP_ERR_STATE without a prior solve.  Changes the internal iterate
 * (not the stored solution). */
int lp_profile_kernels(lp_problem *lp, int32_t reps, double *out);

/* The grid engine's tile shapes after the last lp_solve (no counterpart in
 * the paper: the autotuner of the warp-tile layout).  out[0], out[1]: the
 * candidate index used for the rows of A (the dual kernel) and of A^T (the
 * primal kernel); out[2]: 1 if that solve measured the candidates, 0 if the
 * shapes came from the cache, the default or the options; then per
 * candidate c: out[3 + 4c] run_max, out[4 + 4c] tile_nnz, out[5 + 4c] and
 * out[6 + 4c] the mean ms of the dual and the primal kernel under it (0 when
 * not measured).  cap: doubles available (LP_ERR_INVALID if too few);
 * *count: doubles written.  LP_ERR_STATE without a grid-engine solve. */
int lp_get_tile_tuning(const lp_problem *lp, double *out, int32_t cap, int32_t *count);

/* Forget the autotuners' cached tile shapes: the grid engine's (the next
 * solve of each size class measures again) and the batched path's classes
 * (lp_server_tile_tuning; later requests try the shapes again). */
void lp_tile_cache_clear(void);

void lp_destroy(lp_problem *lp);

/* Power-iteration estimate of ||A||_2 that allocates no memory (the paper
 * has no counterpart; it is the step-size estimate lp_solve computes, as a
 * stand-alone call).  For callers that cannot allocate device memory where
 * they need it: a process that reserved the GPU's memory for its own pool,
 * or a latency-critical path where a cudaMalloc -- which can synchronize the
 * device or fail on a fragmented heap -- is not allowed.
 *   m, n        rows and columns of A; requires m + 2 n <= 1047551
 *               (LP_ERR_INVALID with a message otherwise)
 *   a_*         CSR of A on the device: row_ptr (m + 1), col_idx, val
 *   at_*        CSR of A^T on the device (n + 1 row pointers)
 *   iters       power iterations (lp_solve uses 100); start vector
 *               1/sqrt(n), v <- A^T A v / ||.||, estimate ||A v||; a step
 *               giving zero continues from v_j = (0.5 + h(j) / 2^32) /
 *               sqrt(n), h(j) = j * 2654435761 mod 2^32
 *   stream      cudaStream_t the kernels run on (NULL: legacy stream)
 *   norm_out    host double that receives the estimate (0 if m or n is 0)
 * All work vectors live in one file-scope device array of 2^20 doubles
 * (8 MiB) that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address (a
 * one-time set-up per device, repeated only if the device's context has
 * been replaced, e.g. after cudaDeviceReset): make the first call before
 * any stream capture.  m + 2 n must be at most 1,047,551 (else
 * LP_ERR_INVALID); m = 0 or n = 0 gives 0 without touching the GPU.  Every
 * call shares the array and it keeps the last call's contents; calls that
 * overlap on the GPU (other streams, other threads) race on it.  The call
 * returns after synchronizing `stream`. */
int lp_power_norm_static(int32_t m, int32_t n, const int32_t *a_row_ptr,
                         const int32_t *a_col_idx, const double *a_val,
                         const int32_t *at_row_ptr, const int32_t *at_col_idx,
                         const double *at_val, int32_t iters, void *stream,
                         double *norm_out);

/* ---- batched solving and continuous-batching server ------------------ */

/* A server holds up to hbm_budget_bytes of device memory (allocated once),
 * packs admitted problems into slots of a persistent segmented batch and
 * runs them.  Slots are grouped in four size buckets (by nonzeros); each
 * bucket has its own stream and launch loop, so small problems never wait
 * for large ones.  One bucket launch gives every live slot of the bucket at
 * least one block of check_every iterations and keeps going while the
 * launch's device time budget lasts; finished slots are retired and their
 * memory refilled from the queue between launches.  Requests with at least
 * solo_nnz nonzeros (default 500,000) instead run the single-LP grid path
 * on their own stream, with device memory from the same budget, at most
 * solo_max (default 3) at once.  `opts` applies to every request
 * (precision, eps_rel, ...).  worker: 1 = a background host thread drives
 * the device loop; 0 = the caller drives it through lp_server_pump.
 * Errors: LP_ERR_BUDGET when the budget is below 1 MiB or cannot hold the
 * slot tables for 4,096 slots, before any device work; LP_ERR_OOM when the
 * budget cannot be allocated; LP_ERR_CUDA when a CUDA call fails.  On any
 * error *out is NULL and whatever was created is released. */
int lp_server_create(size_t hbm_budget_bytes, const lp_device_ctx *dev,
                     const lp_solve_opts *opts, int32_t worker, lp_server **out);

/* Queue a problem (its current, possibly presolved LP).  The server borrows
 * `lp` until its result has been polled; the polled answer is also stored in
 * `lp` (lp_get_solution / lp_postsolve work on it).  A problem whose presolve
 * proved it infeasible or unbounded is answered at once (termination
 * LP_INFEASIBLE / LP_UNBOUNDED, no device work).  Fails LP_ERR_BUDGET if the
 * problem alone exceeds the budget.  Several threads may submit to one
 * server at once: a request's device layout is built on its submitting
 * thread, outside the server's lock. */
int lp_batch_submit(lp_server *srv, lp_problem *lp, uint64_t *ticket);

/* LP_PENDING while in flight; LP_OK once done: res, x (n), y (m) of the
 * current LP are filled (pointers may be NULL) and the ticket is released. */
int lp_batch_poll(lp_server *srv, uint64_t ticket, lp_result *res, double *x, double *y);

/* Drive the device loop (worker = 0) for at most `periods` scheduler steps.
 * A step waits for the oldest bucket launch in flight (if any), retires what
 * it finished, admits queued requests and starts a launch for every idle
 * bucket with live slots; launches may still be running when it returns.
 * Returns the number of requests still queued or running. */
int lp_server_pump(lp_server *srv, int32_t periods);

/* Scheduler settings; call before submitting.  solo_nnz > 0: the nonzero
 * count from which a request runs on the single-LP path (<= 0: keep);
 * solo_max in [1, 64]: solo requests running at once (negative: keep);
 * launch_ms in (0, 1000]: device time budget of one bucket launch (default
 * 2 ms; <= 0: keep).  LP_ERR_INVALID for values out of range. */
int lp_server_tune(lp_server *srv, int64_t solo_nnz, int32_t solo_max, double launch_ms);

/* Cancel a queued or running request: its poll returns LP_OK with
 * termination LP_CANCELLED. */
int lp_batch_cancel(lp_server *srv, uint64_t ticket);

/* Statistics (12 int64): out[0] admitted, out[1] finished, out[2] bucket
 * launches, out[3] peak resident bytes, out[4] kernel launches, out[5] queue
 * length, out[6..9] shape index the autotuner uses for each size bucket
 * (nonzeros < 16Ki, < 128Ki, < 1Mi, larger), out[10] host nanoseconds spent
 * issuing bucket launches (order copy, events, the launch, the state
 * read-back), out[11] device nanoseconds of the completed bucket launches. */
int lp_server_stats(const lp_server *srv, int64_t *out);

/* CUDA-graph statistics of the bucket launches (2 int64): out[0] launches
 * replayed from a graph, out[1] graphs instantiated.  With use_graph = 1 (the
 * default) every bucket launch -- the order copy, events, k_batch and the
 * state read-back -- replays a graph instantiated once per bucket and
 * cluster x CTA shape, its copy sizes and the kernel's grid and slot count
 * updated in place; use_graph = 0 issues the same work directly.  The paper
 * has no counterpart (serving is this library's). */
int lp_server_graph_stats(const lp_server *srv, int64_t *out);

/* The batched path's tile-shape autotuner (the paper has no counterpart),
 * one table per process and precision (lp_tile_cache_clear empties it).
 * Requests are classed by m bucket = floor(log2 m / 2) and row-length bucket
 * = floor(log2(nnz / m)); while a class is trying, its packed requests get
 * the shapes 0..5 in turn -- entries per lane {8, 16, 32} x nonzeros per warp
 * tile {512, 2048}, shape c = (entries index) * 2 + (2048 ? 1 : 0) -- and
 * each finished one's device time per nonzero-iteration is recorded; when
 * every shape has 2 samples the class keeps the least mean.  out: *nclasses
 * rows of 15 doubles: m bucket, row-length bucket, chosen shape (-1: still
 * trying), mean ns per nonzero-iteration of shapes 0..5 (-1: no sample),
 * samples of shapes 0..5.  cap: rows out holds (LP_ERR_INVALID, with
 * *nclasses set, if too small). */
int lp_server_tile_tuning(const lp_server *srv, double *out, int32_t cap, int32_t *nclasses);

void lp_server_destroy(lp_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LP_H */
