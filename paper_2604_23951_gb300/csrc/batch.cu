// Batched PDHG and the continuous-batching server (lp_server_* / lp_batch_*).
//
// Many independent LPs ("slots") live in one device arena sized by the
// server's HBM budget.  One persistent launch processes every live slot of a
// size bucket: a thread-block cluster of CL CTAs owns one slot at a time and
// runs K iterations of the same restarted reflected Halpern PDHG as the
// single-LP path (one check iteration, then K - 1 plain ones), with
// cluster.sync() between the phases (A^T y + primal epilogue, A xbar + dual
// epilogue, the check's two KKT products, the decision, the restart copy).
// Reductions are deterministic: warp trees, then the warps of a CTA in
// order, then the CTAs of the cluster in rank order through distributed
// shared memory.  A slot's first launch also runs its set-up (Ruiz +
// Pock-Chambolle scaling, the power iteration for the step, omega_0,
// initial point).  Between launches the host retires finished slots, copies
// their results out and admits queued requests into the freed arena space:
// requests that arrive while others run are admitted as memory frees up and
// their iterations overlap on the device.
//
// Precision: LP_MIXED runs the iteration SpMV on FP32 values times the
// float pairs of the gathered vector with compensated FP32 sums, and keeps
// the set-up, iterates, anchor, epilogues, reductions and decisions in FP64;
// LP_FP64 runs everything in FP64.  KKT checks always use the FP64 scaled
// matrix.
//
// Autotuner: for each size bucket (by nonzeros) the server times the
// candidate (cluster size, CTA size) shapes on its first launches and keeps
// the fastest per nonzero-iteration.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "lp_internal.h"
#include "layout.h"
#include "pdhg_epi.cuh"
#include "pdhg_state.cuh"
#include "spmv_warp.cuh"

namespace cg = cooperative_groups;

namespace gb300lp {

void set_last_error(const std::string &m);
const HostLP &problem_current(const lp_problem *lp);
int problem_proven_status(const lp_problem *lp);
constexpr long long kSoloNnz = 500000;  // larger requests run on the single-LP grid path
void problem_store_solution(lp_problem *lp, const std::vector<double> &x,
                            const std::vector<double> &y, const std::vector<double> &z);
double problem_original_kkt(const lp_problem *lp, const double *x, const double *y,
                            const double *z);

constexpr int ST_SETUP = -2;
constexpr int kMaxCluster = 8;
constexpr int kMaxWarps = 16;  // CTAs of up to 512 threads

// One slot's device layout: A and A^T renumbered and cut into warp tiles as
// in the single-LP path (layout.h), so vectors are in the permuted order.
struct SlotDesc {
  int m, n;
  long long nnz;
  int a_ntiles, a_nlong, t_ntiles, t_nlong;
  const int2 *a_tiles, *t_tiles;
  const int *a_rp, *a_ci, *t_rp, *t_ci;
  const double *a_v0, *t_v0;
  double *a_v, *t_v;
  float *a_vf, *t_vf;
  const double *c0, *lx0, *ux0, *lc0, *uc0, *pv0;
  double *c, *lx, *ux, *lc, *uc;
  double *dr, *dc, *dr2, *dc2, *idr, *idc;
  double *x, *x0, *xbar, *xhat, *y, *y0, *yhat;
  float2 *xbarf, *yf;  // mixed: x-bar and y as float pairs (split_f2)
  double *xout, *yout, *zout;
  const double *xinit, *yinit;  // warm start (unscaled, device order) or NULL
};

struct BatchConst {
  int K, ruiz_iters, pock_chambolle, power_iters;
  int infeas_every;
  long long max_iter;
  double step_size, primal_weight;
  long long budget_ns;  // device time a launch gives its slots (>= one block of K each)
};

// ---------------------------------------------------------------------------
// device helpers

// control words of the slot a cluster is working on; every CTA keeps its own
// copy in shared memory, written by rank 0 through distributed shared memory
// before a cluster barrier, so every control-flow decision is read from the
// CTA's own shared memory and is identical across the cluster
struct Ctl {
  int status, restart_flag, k_base, k_off, halpern, mixed_active;
  long long t;
  double tau, sigma, rho;
};

struct BatchShared {
  double redd[kMaxWarps];  // whole-CTA rows of the warp engine
  F2 red2[kMaxWarps];  // the same for the compensated FP32 SpMV
  double wsum[kMaxWarps][NQ];
  double part[kMaxCluster][NQ];  // used on rank 0
  double total[NQ];
  Ctl ctl;
  double bcast;
  int cont;
};

// thread 0 of a CTA: read the slot's control words from global memory
// (volatile: no stale L1 copy); the caller synchronizes the CTA
__device__ __forceinline__ void load_ctl(const State *st, Ctl &c) {
  const volatile State *v = st;
  c.status = v->status;
  c.restart_flag = v->restart_flag;
  c.k_base = v->k_base;
  c.k_off = v->k_off;
  c.halpern = v->halpern;
  c.mixed_active = v->mixed_active;
  c.t = v->t;
  c.tau = v->tau;
  c.sigma = v->sigma;
  c.rho = v->rho;
}

// rank 0 thread 0, after updating *st: copy its control words into the
// shared memory of every CTA of the cluster (the caller then syncs the cluster)
__device__ __forceinline__ void bcast_ctl(const State *st, BatchShared &sh,
                                          cg::cluster_group &cl) {
  Ctl c;
  c.status = st->status;
  c.restart_flag = st->restart_flag;
  c.k_base = st->k_base;
  c.k_off = st->k_off;
  c.halpern = st->halpern;
  c.mixed_active = st->mixed_active;
  c.t = st->t;
  c.tau = st->tau;
  c.sigma = st->sigma;
  c.rho = st->rho;
  for (int r = 0; r < (int)cl.num_blocks(); ++r) cl.map_shared_rank(&sh, r)->ctl = c;
}

__device__ __forceinline__ Halpern halpern_ctl(const Ctl &c, int j) {
  double lam = 1.0;
  if (c.halpern) {
    int k = (j == 0) ? c.k_base : c.k_off + j;
    lam = (k + 1.0) / (k + 2.0);
  }
  Halpern h;
  h.a = lam * (1.0 + c.rho);
  h.b = -lam * c.rho;
  h.g = 1.0 - lam;
  return h;
}

// Deterministic cluster-wide sum of acc[0..nq) (quantity ids qid[]); the
// result lands in sh.total[qid[q]] of rank 0 (returned to rank 0 thread 0).
template <int NQL>
__device__ __forceinline__ void cluster_sum(const double (&acc)[NQL], const int (&qid)[NQL],
                                            BatchShared &sh, cg::cluster_group &cl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQL; ++q) {
    double v = warp_sum(acc[q]);
    if (lane == 0) sh.wsum[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQL) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh.wsum[w][threadIdx.x];
    BatchShared *r0 = cl.map_shared_rank(&sh, 0);
    r0->part[cl.block_rank()][threadIdx.x] = s;
  }
  cl.sync();
  if (cl.block_rank() == 0 && threadIdx.x < NQL) {
    double s = 0.0;
    for (int r = 0; r < (int)cl.num_blocks(); ++r) s += sh.part[r][threadIdx.x];
    sh.total[qid[threadIdx.x]] = s;
  }
  __syncthreads();
}

// one Ruiz / Pock-Chambolle pass over the rows of a matrix: dnew[r] =
// dself[r] / sqrt(max or sum_k (dr |a|) dc)
template <bool TRANSPOSED, bool SUM>
__device__ __forceinline__ void scale_rows(int rows, const int *rp, const int *ci,
                                           const double *a0, const double *dself,
                                           const double *dother, double *dnew, int gt,
                                           int gs) {
  for (int r = gt; r < rows; r += gs) {
    const double ds = dself[r];
    double acc = 0.0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      const double v = TRANSPOSED ? (dother[ci[k]] * fabs(a0[k])) * ds
                                  : (ds * fabs(a0[k])) * dother[ci[k]];
      acc = SUM ? acc + v : (v > acc ? v : acc);
    }
    dnew[r] = acc > 0.0 ? ds / sqrt(acc) : ds;
  }
}

// ---------------------------------------------------------------------------
// set-up of one slot (scaling, step size, primal weight, initial point)

// Both precisions set up in FP64 (scaling, power iteration): the mixed mode
// differs only in its iteration SpMV, as on the grid engine.
template <bool MIXED>
__device__ void slot_setup(const SlotDesc &D, State *st, const BatchConst &C, BatchShared &sh,
                           cg::cluster_group &cl) {
  const int m = D.m, n = D.n;
  const int gt = cl.block_rank() * blockDim.x + threadIdx.x;
  const int gs = cl.num_blocks() * blockDim.x;
  double *dr = D.dr, *dc = D.dc, *dr2 = D.dr2, *dc2 = D.dc2;
  for (int i = gt; i < m; i += gs) dr[i] = 1.0;
  for (int j = gt; j < n; j += gs) dc[j] = 1.0;
  cl.sync();
  for (int it = 0; it < C.ruiz_iters; ++it) {
    scale_rows<false, false>(m, D.a_rp, D.a_ci, D.a_v0, dr, dc, dr2, gt, gs);
    scale_rows<true, false>(n, D.t_rp, D.t_ci, D.t_v0, dc, dr, dc2, gt, gs);
    cl.sync();
    double *t = dr; dr = dr2; dr2 = t;
    t = dc; dc = dc2; dc2 = t;
  }
  if (C.pock_chambolle) {
    scale_rows<false, true>(m, D.a_rp, D.a_ci, D.a_v0, dr, dc, dr2, gt, gs);
    scale_rows<true, true>(n, D.t_rp, D.t_ci, D.t_v0, dc, dr, dc2, gt, gs);
    cl.sync();
    double *t = dr; dr = dr2; dr2 = t;
    t = dc; dc = dc2; dc2 = t;
  }
  if (dr != D.dr) {
    for (int i = gt; i < m; i += gs) D.dr[i] = dr[i];
    for (int j = gt; j < n; j += gs) D.dc[j] = dc[j];
    cl.sync();
  }
  dr = D.dr;
  dc = D.dc;
  // scaled problem; norms of c~ and bhat~
  double acc[2] = {0.0, 0.0};
  for (int i = gt; i < m; i += gs) {
    const double d = dr[i];
    for (int k = D.a_rp[i]; k < D.a_rp[i + 1]; ++k) {
      const double v = (d * D.a_v0[k]) * dc[D.a_ci[k]];
      D.a_v[k] = v;
      if (MIXED) D.a_vf[k] = (float)v;
    }
    D.idr[i] = 1.0 / d;
    const double l = d * D.lc0[i], u = d * D.uc0[i];
    D.lc[i] = l;
    D.uc[i] = u;
    const bool lf = isfinite(l), uf = isfinite(u);
    if (lf) acc[1] += l * l;
    if (uf && !(lf && l == u)) acc[1] += u * u;
  }
  for (int j = gt; j < n; j += gs) {
    const double d = dc[j];
    for (int k = D.t_rp[j]; k < D.t_rp[j + 1]; ++k) {
      const double v = (dr[D.t_ci[k]] * D.t_v0[k]) * d;
      D.t_v[k] = v;
      if (MIXED) D.t_vf[k] = (float)v;
    }
    D.idc[j] = 1.0 / d;
    const double cj = d * D.c0[j];
    D.c[j] = cj;
    D.lx[j] = D.lx0[j] / d;
    D.ux[j] = D.ux0[j] / d;
    acc[0] += cj * cj;
  }
  {
    const int qid[2] = {Q_CN, Q_BN};
    cluster_sum<2>(acc, qid, sh, cl);
  }
  // power iteration on A~^T A~ (v in xhat, u in yhat, w in xbar)
  double eta = C.step_size;
  if (!(eta > 0.0)) {
    double pw = 0.0;
    if (m > 0 && n > 0) {
      const double v0 = 1.0 / sqrt((double)n);
      for (int j = gt; j < n; j += gs) {
        D.xhat[j] = v0;
      }
      cl.sync();
      const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
      for (int it = 0; it <= C.power_iters; ++it) {
        // u = A~ v
        double a2[1] = {0.0};
        {
          StoreSqEpi<double> e{D.yhat, 0.0};
          warp_spmv<double, double, double>(D.a_nlong, D.a_tiles, D.a_ntiles, D.a_rp, D.a_ci,
                                            D.a_v, D.xhat, e, sh.redd, rank, CL);
          a2[0] = e.acc;
        }
        if (it == C.power_iters) {
          const int qid[1] = {Q_PW};
          cluster_sum<1>(a2, qid, sh, cl);
          if (cl.block_rank() == 0 && threadIdx.x == 0) pw = sqrt(sh.total[Q_PW]);
          break;
        }
        cl.sync();
        // w = A~^T u
        {
          StoreSqEpi<double> e{D.xbar, 0.0};
          warp_spmv<double, double, double>(D.t_nlong, D.t_tiles, D.t_ntiles, D.t_rp, D.t_ci,
                                            D.t_v, D.yhat, e, sh.redd, rank, CL);
          a2[0] = e.acc;
        }
        const int qid[1] = {Q_PW};
        cluster_sum<1>(a2, qid, sh, cl);
        // broadcast ||w|| to every CTA's shared memory
        if (cl.block_rank() == 0 && threadIdx.x == 0) {
          const double nwv = sqrt(sh.total[Q_PW]);
          for (int r = 0; r < (int)cl.num_blocks(); ++r) cl.map_shared_rank(&sh, r)->bcast = nwv;
        }
        cl.sync();
        const double nw = sh.bcast;
        // a zero w continues from the fallback start vector
        for (int j = gt; j < n; j += gs) {
          D.xhat[j] = nw > 0.0 ? D.xbar[j] / nw : D.pv0[j];
        }
        cl.sync();
      }
    }
    if (cl.block_rank() == 0 && threadIdx.x == 0) eta = pw > 0.0 ? 0.998 / pw : 1.0;
  }
  // initial point (projected zero, or the warm start) and state
  for (int j = gt; j < n; j += gs) {
    const double v = D.xinit ? D.xinit[j] / dc[j] : clampd(0.0, D.lx[j], D.ux[j]);
    D.x[j] = v;
    D.x0[j] = v;
  }
  for (int i = gt; i < m; i += gs) {
    const double v = D.yinit ? D.yinit[i] / dr[i] : 0.0;
    D.y[i] = v;
    D.y0[i] = v;
    if (MIXED) D.yf[i] = split_f2(v);
  }
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    const double cn = sqrt(sh.total[Q_CN]), bn = sqrt(sh.total[Q_BN]);
    const double om = C.primal_weight > 0 ? C.primal_weight : ((cn > 0 && bn > 0) ? cn / bn : 1.0);
    st->eta = eta;
    st->omega = om;
    st->omega0 = om;
    st->tau = eta / om;
    st->sigma = eta * om;
    st->t = 0;
    st->iters = 0;
    st->k_base = 0;
    st->k_off = 0;
    st->restarts = 0;
    st->restart_flag = 0;
    st->r0 = st->r_prev = st->last_r = 0.0;
    st->rel_kkt = INFINITY;
    st->status = ST_RUNNING;
    bcast_ctl(st, sh, cl);
  }
  cl.sync();
}

// ---------------------------------------------------------------------------
// K iterations of one slot

// K1 (rows of A^T) or K2 (rows of A) with the shared epilogues; f32 selects
// the FP32 SpMV of the mixed mode
template <bool CHECK>
__device__ __forceinline__ void phase_primal(const SlotDesc &D, bool f32, double tau,
                                             const Halpern &hc, BatchShared &sh, int rank, int CL,
                                             double (&acc)[10]) {
  if (f32) {
    PrimalEpi<CHECK, true> e{D.c, D.lx, D.ux, D.x, D.x0, D.xbar, D.xhat, D.xbarf, tau, hc,
                             0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    warp_spmv<float, float2, F2>(D.t_nlong, D.t_tiles, D.t_ntiles, D.t_rp, D.t_ci, D.t_vf, D.yf,
                                 e, sh.red2, rank, CL);
    acc[0] = e.acc0;
    acc[1] = e.acc1;
  } else {
    PrimalEpi<CHECK, false> e{D.c, D.lx, D.ux, D.x, D.x0, D.xbar, D.xhat, D.xbarf, tau, hc,
                              0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    warp_spmv<double, double, double>(D.t_nlong, D.t_tiles, D.t_ntiles, D.t_rp, D.t_ci, D.t_v,
                                      D.y, e, sh.redd, rank, CL);
    acc[0] = e.acc0;
    acc[1] = e.acc1;
  }
}

template <bool CHECK>
__device__ __forceinline__ void phase_dual(const SlotDesc &D, bool f32, double sigma,
                                           const Halpern &hc, BatchShared &sh, int rank, int CL,
                                           double (&acc)[10]) {
  if (f32) {
    DualEpi<CHECK, true> e{D.lc, D.uc, D.y, D.y0, D.yhat, D.yf, sigma, hc,
                           0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    warp_spmv<float, float2, F2>(D.a_nlong, D.a_tiles, D.a_ntiles, D.a_rp, D.a_ci, D.a_vf,
                                 D.xbarf, e, sh.red2, rank, CL);
    acc[2] = e.acc0;
    acc[3] = e.acc1;
  } else {
    DualEpi<CHECK, false> e{D.lc, D.uc, D.y, D.y0, D.yhat, D.yf, sigma, hc,
                            0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    warp_spmv<double, double, double>(D.a_nlong, D.a_tiles, D.a_ntiles, D.a_rp, D.a_ci, D.a_v,
                                      D.xbar, e, sh.redd, rank, CL);
    acc[2] = e.acc0;
    acc[3] = e.acc1;
  }
}

// K3 (the KKT products of the check, FP64 scaled matrix, unscaled
// quantities) and the cluster-wide sum of acc[0..10) into sh.total (rank 0)
__device__ __forceinline__ void slot_kkt(const SlotDesc &D, BatchShared &sh,
                                         cg::cluster_group &cl, double (&acc)[10], bool inf) {
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  {
    KktRowEpi e{D.dr, D.idr, D.lc0, D.uc0, D.yhat, 0.0, 0.0, 0.0};
    warp_spmv<double, double, double>(D.a_nlong, D.a_tiles, D.a_ntiles, D.a_rp, D.a_ci, D.a_v,
                                      D.xhat, e, sh.redd, rank, CL);
    acc[4] = e.rp2;
    acc[5] = e.rdy2;
    acc[6] = e.dy;
  }
  {
    KktColEpi e{D.c, D.dc, D.idc, D.c0, D.lx0, D.ux0, D.xhat, D.zout, 0.0, 0.0, 0.0};
    warp_spmv<double, double, double>(D.t_nlong, D.t_tiles, D.t_ntiles, D.t_rp, D.t_ci, D.t_v,
                                      D.yhat, e, sh.redd, rank, CL);
    acc[7] = e.rd2;
    acc[8] = e.dl;
    acc[9] = e.p;
  }
  const int qid[10] = {Q_XRES, Q_XD, Q_YRES, Q_YD, Q_RP, Q_RDY, Q_DY, Q_RD, Q_DL, Q_P};
  cluster_sum<10>(acc, qid, sh, cl);
  if (inf) {
    // infeasibility test of the direction (xh - x0, yh - y0): xbar (free
    // after K2) holds d~, yout (written only at the end) the projected w~
    const int gt = rank * blockDim.x + threadIdx.x, gs = CL * blockDim.x;
    double ia[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = gt; j < D.n; j += gs)
      inf_col_prep(j, D.xhat, D.x0, D.dc, D.c0, D.lx0, D.ux0, D.xbar, ia[0], ia[1]);
    cl.sync();
    {
      InfRowEpi e{D.dr, D.idr, D.lc0, D.uc0, D.yhat, D.y0, D.yout, 0.0, 0.0};
      warp_spmv<double, double, double>(D.a_nlong, D.a_tiles, D.a_ntiles, D.a_rp, D.a_ci,
                                        D.a_v, D.xbar, e, sh.redd, rank, CL);
      ia[2] = e.v2;
      ia[3] = e.dobj;
    }
    cl.sync();
    {
      InfColEpi e{D.idc, D.lx0, D.ux0, 0.0, 0.0};
      warp_spmv<double, double, double>(D.t_nlong, D.t_tiles, D.t_ntiles, D.t_rp, D.t_ci,
                                        D.t_v, D.yout, e, sh.redd, rank, CL);
      ia[4] = e.r2;
      ia[5] = e.dobj;
    }
    const int iq[6] = {Q_ICD, Q_IPVC, Q_IPVR, Q_IDOR, Q_IDR, Q_IDOC};
    cluster_sum<6>(ia, iq, sh, cl);
  }
}

// One block of iterations t0 .. t0 + K - 1 (t0 = iterations done, a multiple
// of K): the first is the check iteration.  When max_iter falls inside the
// block, the block stops there: its last iteration also writes T(z), which
// is evaluated (KKT, LP_ITER_LIMIT) -- the single-LP path's semantics.
template <bool MIXED>
__device__ void slot_iterate(const SlotDesc &D, State *st, const BatchConst &C, BatchShared &sh,
                             cg::cluster_group &cl) {
  const int m = D.m, n = D.n;
  const int gt = cl.block_rank() * blockDim.x + threadIdx.x;
  const int gs = cl.num_blocks() * blockDim.x;
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  const long long rem = C.max_iter - sh.ctl.t;
  if (rem <= 0) {
    // defensive: nothing left to run; keep the last check's point
    cl.sync();
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
      st->status = 1;
      st->iters = st->t;
      bcast_ctl(st, sh, cl);
    }
    cl.sync();
    return;
  }
  const int jmax = rem < C.K ? (int)rem : C.K;
  const bool final_block = rem <= C.K;
  for (int j = 0; j < jmax; ++j) {
    if (sh.ctl.status != ST_RUNNING) break;
    const bool check = (j == 0);
    const bool last = final_block && j == jmax - 1;
    const bool hats = check || last;
    const Halpern hc = halpern_ctl(sh.ctl, j);
    const double tau = sh.ctl.tau, sigma = sh.ctl.sigma;
    const bool f32 = MIXED && sh.ctl.mixed_active;  // FP32 SpMV until the FP64 switch
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // K1: rows of A^T
    if (hats) phase_primal<true>(D, f32, tau, hc, sh, rank, CL, acc);
    else phase_primal<false>(D, f32, tau, hc, sh, rank, CL, acc);
    cl.sync();
    // K2: rows of A
    if (hats) phase_dual<true>(D, f32, sigma, hc, sh, rank, CL, acc);
    else phase_dual<false>(D, f32, sigma, hc, sh, rank, CL, acc);
    cl.sync();
    if (check) {
      slot_kkt(D, sh, cl, acc, infeas_due(sh.ctl.t, C.K, C.infeas_every));
      if (cl.block_rank() == 0 && threadIdx.x == 0) {
        check_update(st, sh.total, false);
        bcast_ctl(st, sh, cl);
      }
      cl.sync();
      if (sh.ctl.status != ST_RUNNING) break;
      if (sh.ctl.restart_flag) {
        for (int c = gt; c < n; c += gs) {
          const double v = D.xhat[c];
          D.x[c] = v;
          D.x0[c] = v;
        }
        for (int r = gt; r < m; r += gs) {
          const double v = D.yhat[r];
          D.y[r] = v;
          D.y0[r] = v;
          if (MIXED) D.yf[r] = split_f2(v);
        }
        cl.sync();
      }
    }
    if (last) {
      // max_iter reached: evaluate the last T(z)
      double acc2[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      slot_kkt(D, sh, cl, acc2, false);
      if (cl.block_rank() == 0 && threadIdx.x == 0) {
        check_update(st, sh.total, true);
        st->iters = C.max_iter;
        bcast_ctl(st, sh, cl);
      }
      cl.sync();
    }
  }
  // finished slots: unscaled answer (the last T(z) evaluated)
  if (sh.ctl.status != ST_RUNNING && sh.ctl.status != ST_SETUP) {
    for (int c = gt; c < n; c += gs) D.xout[c] = D.dc[c] * D.xhat[c];
    for (int r = gt; r < m; r += gs) D.yout[r] = D.dr[r] * D.yhat[r];
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One launch over the slots order[0..nord): each cluster takes slots
// cid, cid + ncl, ...; a slot runs blocks of K iterations until it finishes
// or its share of the launch's time budget is spent (at least one block).
// On leaving a slot, rank 0 copies its state to sout[oi] for the host.
template <bool MIXED>
__global__ void __launch_bounds__(512, 1) k_batch(const SlotDesc *__restrict__ desc, State *states,
                                               const int *__restrict__ order, int nord,
                                               State *sout, BatchConst C) {
  __shared__ BatchShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks();
  const int ncl = gridDim.x / CL;
  const int cid = blockIdx.x / CL;
  const bool lead = cl.block_rank() == 0 && threadIdx.x == 0;
  const int rounds = (nord + ncl - 1) / ncl;
  const long long share = C.budget_ns / (rounds > 0 ? rounds : 1);
  for (int oi = cid; oi < nord; oi += ncl) {
    const int s = order[oi];
    const SlotDesc &D = desc[s];
    State *st = states + s;
    // the slot's state was written by an earlier launch: every CTA reads the
    // same control words
    if (threadIdx.x == 0) load_ctl(st, sh.ctl);
    __syncthreads();
    const unsigned long long t0 = lead ? global_ns() : 0ull;
    if (sh.ctl.status == ST_SETUP) slot_setup<MIXED>(D, st, C, sh, cl);
    while (sh.ctl.status == ST_RUNNING) {
      slot_iterate<MIXED>(D, st, C, sh, cl);
      if (lead) {
        const int go = sh.ctl.status == ST_RUNNING && (long long)(global_ns() - t0) < share;
        for (int r = 0; r < CL; ++r) cl.map_shared_rank(&sh, r)->cont = go;
      }
      cl.sync();
      if (!sh.cont) break;
    }
    if (lead) {
      st->dev_ns += (long long)(global_ns() - t0);
      sout[oi] = *st;
    }
    cl.sync();
  }
}

// ---------------------------------------------------------------------------
// host side: arena, slots, autotuner, server loop

struct Shape {
  int cl, block;
};

static const Shape kShapes[] = {{1, 128}, {1, 256}, {2, 256}, {4, 256}, {8, 256}, {8, 512}};
constexpr int kNumBuckets = 4;

static int bucket_of(long long nnz) {
  if (nnz < 16384) return 0;
  if (nnz < 131072) return 1;
  if (nnz < 1048576) return 2;
  return 3;
}

// candidate shapes per bucket (indices into kShapes)
static std::vector<int> candidates(int bucket) {
  switch (bucket) {
    case 0: return {0, 1};
    case 1: return {0, 1, 2};
    case 2: return {1, 2, 3, 4};
    default: return {3, 4, 5};
  }
}

struct Tuner {
  std::vector<int> cand;
  std::vector<double> best_ns;  // per candidate: best ns per nonzero-iteration
  int next = 0;
  int chosen = -1;
  int trials = 0;
  Shape pick() {
    if (chosen >= 0) return kShapes[chosen];
    return kShapes[cand[next]];
  }
  int current() const { return chosen >= 0 ? chosen : cand[next]; }
  void record(double ns_per_nnz_iter) {
    if (chosen >= 0) return;
    best_ns[next] = std::min(best_ns[next], ns_per_nnz_iter);
    ++trials;
    next = (next + 1) % (int)cand.size();
    if (trials >= 2 * (int)cand.size()) {
      int b = 0;
      for (int q = 1; q < (int)cand.size(); ++q)
        if (best_ns[q] < best_ns[b]) b = q;
      chosen = cand[b];
    }
  }
};

// Tile-shape autotuner of the batched path.  Requests are classed by
// (m bucket = floor(log2 m / 2), row-length bucket = floor(log2(nnz / m)));
// while a class is trying, its packed requests get the candidate shapes in
// turn -- 8 / 16 / 32 entries per lane x 512 / 2048 nonzeros per warp tile,
// the grid engine's candidates (rows over kCtaRow entries take a whole CTA
// here) -- and each finished slot's device time per nonzero-iteration
// (State::dev_ns, set-up included) is recorded for its shape; once every
// shape has kTileSamples samples the class keeps the one with the least mean.
constexpr int kTileCands = 6;
constexpr int kTileSamples = 2;
static TileShape tile_shape(int c) {
  static const int rm[3] = {8, 16, 32};
  TileShape t;
  t.run_max = rm[c / 2];
  t.tile_nnz = (c & 1) ? 2048 : 512;
  t.segmented = false;
  return t;
}

struct TileClass {
  int next = 0;
  int chosen = -1;
  double sum[kTileCands] = {0, 0, 0, 0, 0, 0};
  int cnt[kTileCands] = {0, 0, 0, 0, 0, 0};
};

// the classes of every server of the process, by precision and class key
// (lp_tile_cache_clear forgets them)
std::mutex g_batch_tile_mu;
std::map<int, TileClass> g_batch_tile;

void batch_tile_cache_clear() {
  std::lock_guard<std::mutex> lk(g_batch_tile_mu);
  g_batch_tile.clear();
}

static int tile_class_key(int m, long long nnz) {
  if (m <= 0) return 0;
  const int mb = (int)std::floor(std::log2((double)m) / 2.0);
  const int lb = (int)std::floor(std::log2(std::max(1.0, (double)nnz / (double)m)));
  return mb * 64 + lb;
}
static int tile_table_key(int precision, int m, long long nnz) {
  return (precision == LP_MIXED ? 1 << 20 : 0) + tile_class_key(m, nnz);
}

// first-fit allocator over [0, size) with coalescing of free ranges
struct RangeAlloc {
  std::map<size_t, size_t> free_;  // offset -> bytes
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
  }
  bool alloc(size_t bytes, size_t &off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        off = it->first;
        size_t rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// host copy of one request, packed in the slot's device layout
struct Packed {
  int m = 0, n = 0;
  long long nnz = 0;
  std::vector<unsigned char> blob;  // bytes copied to the slot's arena block
  size_t bytes = 0;
  SlotDesc rel{};  // pointers as offsets from the block start
  double bnorm = 0, cnorm = 0, off = 0;
  std::vector<int> rperm, cperm;  // device order -> request order
  int tile = 0;             // tile shape candidate (tile_shape)
  bool tile_trial = false;  // packed while its class was trying shapes
};

static size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// xw / yw: NULL, or a warm start (x: n, y: m, unscaled, the request's own
// order) stored with the inputs in the slot's device order
static void pack_request(const HostLP &h, Packed &p, const double *xw = nullptr,
                         const double *yw = nullptr, TileShape shape = TileShape{}) {
  Layout L;
  shape.segmented = false;  // rows over kCtaRow entries take a whole CTA here
  build_layout(h, L, shape);
  p.m = h.m;
  p.n = h.n;
  p.nnz = h.nnz();
  const int m = h.m, n = h.n;
  const long long nnz = h.nnz();
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    size_t o = cur;
    cur += align16(std::max<size_t>(bytes, 16));
    return o;
  };
  SlotDesc &r = p.rel;
  auto P = [](size_t o) { return reinterpret_cast<void *>(o); };
  const size_t ntA = L.pA.tiles.size(), ntT = L.pT.tiles.size();
  const size_t nzA = (size_t)nnz, nzT = (size_t)nnz;
  size_t o_tA = take(sizeof(int2) * ntA), o_tT = take(sizeof(int2) * ntT);
  size_t o_arp = take(sizeof(int) * (m + 1)), o_aci = take(sizeof(int) * nzA);
  size_t o_trp = take(sizeof(int) * (n + 1)), o_tci = take(sizeof(int) * nzT);
  size_t o_av0 = take(8 * nzA), o_tv0 = take(8 * nzT), o_av = take(8 * nzA), o_tv = take(8 * nzT);
  size_t o_avf = take(4 * nzA), o_tvf = take(4 * nzT);
  size_t o_c0 = take(8 * n), o_lx0 = take(8 * n), o_ux0 = take(8 * n);
  size_t o_lc0 = take(8 * m), o_uc0 = take(8 * m), o_pv0 = take(8 * n);
  const bool warm = xw || yw;
  size_t o_xi = warm ? take(8 * n) : 0, o_yi = warm ? take(8 * m) : 0;
  r.m = m;
  r.n = n;
  r.nnz = nnz;
  r.a_ntiles = (int)ntA;
  r.t_ntiles = (int)ntT;
  r.a_nlong = L.pA.nlong;
  r.t_nlong = L.pT.nlong;
  r.a_tiles = (const int2 *)P(o_tA);
  r.t_tiles = (const int2 *)P(o_tT);
  r.a_rp = (const int *)P(o_arp);
  r.a_ci = (const int *)P(o_aci);
  r.t_rp = (const int *)P(o_trp);
  r.t_ci = (const int *)P(o_tci);
  r.a_v0 = (const double *)P(o_av0);
  r.t_v0 = (const double *)P(o_tv0);
  r.a_v = (double *)P(o_av);
  r.t_v = (double *)P(o_tv);
  r.a_vf = (float *)P(o_avf);
  r.t_vf = (float *)P(o_tvf);
  r.c0 = (const double *)P(o_c0);
  r.lx0 = (const double *)P(o_lx0);
  r.ux0 = (const double *)P(o_ux0);
  r.lc0 = (const double *)P(o_lc0);
  r.uc0 = (const double *)P(o_uc0);
  r.pv0 = (const double *)P(o_pv0);
  r.xinit = warm ? (const double *)P(o_xi) : nullptr;
  r.yinit = warm ? (const double *)P(o_yi) : nullptr;
  const size_t input_end = cur;
  double **colv[] = {&r.c, &r.lx, &r.ux, &r.dc, &r.dc2, &r.idc, &r.x, &r.x0, &r.xbar, &r.xhat,
                     &r.xout, &r.zout};
  for (double **q : colv) *q = (double *)P(take(8 * n));
  double **rowv[] = {&r.lc, &r.uc, &r.dr, &r.dr2, &r.idr, &r.y, &r.y0, &r.yhat, &r.yout};
  for (double **q : rowv) *q = (double *)P(take(8 * m));
  r.xbarf = (float2 *)P(take(8 * n));
  r.yf = (float2 *)P(take(8 * m));
  p.bytes = align16(cur);
  // the host blob covers the inputs; the rest of the block is device work space
  p.blob.assign(input_end, 0);
  unsigned char *b = p.blob.data();
  auto put = [b](size_t o, const void *src, size_t bytes) {
    if (bytes) std::memcpy(b + o, src, bytes);
  };
  put(o_tA, L.pA.tiles.data(), sizeof(int2) * ntA);
  put(o_tT, L.pT.tiles.data(), sizeof(int2) * ntT);
  put(o_arp, L.arp.data(), sizeof(int) * (m + 1));
  put(o_aci, L.aci.data(), sizeof(int) * nzA);
  put(o_trp, L.trp.data(), sizeof(int) * (n + 1));
  put(o_tci, L.tci.data(), sizeof(int) * nzT);
  put(o_av0, L.av.data(), 8 * nzA);
  put(o_tv0, L.tv.data(), 8 * nzT);
  put(o_c0, L.c0.data(), 8 * n);
  put(o_lx0, L.lx0.data(), 8 * n);
  put(o_ux0, L.ux0.data(), 8 * n);
  put(o_lc0, L.lc0.data(), 8 * m);
  put(o_uc0, L.uc0.data(), 8 * m);
  put(o_pv0, L.pv0.data(), 8 * n);
  if (warm) {
    double *xi = reinterpret_cast<double *>(b + o_xi);
    double *yi = reinterpret_cast<double *>(b + o_yi);
    for (int j = 0; j < n; ++j) xi[j] = xw ? xw[L.cperm[j]] : 0.0;
    for (int i = 0; i < m; ++i) yi[i] = yw ? yw[L.rperm[i]] : 0.0;
  }
  p.bnorm = L.bnorm;
  p.cnorm = L.cnorm;
  p.off = L.off;
  p.rperm = std::move(L.rperm);
  p.cperm = std::move(L.cperm);
}

static SlotDesc relocate(const SlotDesc &rel, unsigned char *base) {
  SlotDesc d = rel;
  auto R = [base](auto p) { return reinterpret_cast<decltype(p)>(base + reinterpret_cast<size_t>(p)); };
  d.a_tiles = R(rel.a_tiles);
  d.t_tiles = R(rel.t_tiles);
  d.idr = R(rel.idr);
  d.idc = R(rel.idc);
  d.a_rp = R(rel.a_rp);
  d.a_ci = R(rel.a_ci);
  d.t_rp = R(rel.t_rp);
  d.t_ci = R(rel.t_ci);
  d.a_v0 = R(rel.a_v0);
  d.t_v0 = R(rel.t_v0);
  d.a_v = R(rel.a_v);
  d.t_v = R(rel.t_v);
  d.a_vf = R(rel.a_vf);
  d.t_vf = R(rel.t_vf);
  d.c0 = R(rel.c0);
  d.lx0 = R(rel.lx0);
  d.ux0 = R(rel.ux0);
  d.lc0 = R(rel.lc0);
  d.uc0 = R(rel.uc0);
  d.pv0 = R(rel.pv0);
  d.xinit = rel.xinit ? R(rel.xinit) : nullptr;
  d.yinit = rel.yinit ? R(rel.yinit) : nullptr;
  d.c = R(rel.c);
  d.lx = R(rel.lx);
  d.ux = R(rel.ux);
  d.lc = R(rel.lc);
  d.uc = R(rel.uc);
  d.dr = R(rel.dr);
  d.dc = R(rel.dc);
  d.dr2 = R(rel.dr2);
  d.dc2 = R(rel.dc2);
  d.x = R(rel.x);
  d.x0 = R(rel.x0);
  d.xbar = R(rel.xbar);
  d.xhat = R(rel.xhat);
  d.y = R(rel.y);
  d.y0 = R(rel.y0);
  d.yhat = R(rel.yhat);
  d.xbarf = R(rel.xbarf);
  d.yf = R(rel.yf);
  d.xout = R(rel.xout);
  d.yout = R(rel.yout);
  d.zout = R(rel.zout);
  return d;
}

struct Request {
  uint64_t ticket = 0;
  lp_problem *lp = nullptr;
  Packed pk;
  bool solo = false;
  size_t solo_bytes = 0;  // arena estimate of a solo request
  double t_submit = 0;    // first submission (a re-solve keeps it)
  bool cancelled = false;
  // a re-solve asked for by the original-LP check: tighter tolerance and a
  // warm start (solo requests; batched ones carry it in pk), the work done
  double eps_rel = -1.0;  // < 0: the server's
  std::vector<double> xw, yw;
  int refinements = 0;
  long long iters_before = 0;
  double solve_s_before = 0;
};

// device bytes the single-LP path allocates for an LP (upper estimate)
static size_t solo_estimate(const HostLP &h) {
  const size_t nz = (size_t)h.nnz() + 64;
  return nz * 2 * (4 + 8 + 8 + 4) + (size_t)h.m * 8 * 16 + (size_t)h.n * 8 * 22 +
         (size_t)(h.m + h.n) * 8 + (size_t(64) << 20);
}

struct Done {
  lp_result res{};
  std::vector<double> x, y, z;
  lp_problem *lp = nullptr;
};

struct Slot {
  bool used = false;
  uint64_t ticket = 0;
  lp_problem *lp = nullptr;
  size_t off = 0, bytes = 0;
  int m = 0, n = 0;
  long long nnz = 0;
  int bucket = 0;
  SlotDesc desc{};
  std::vector<int> rperm, cperm;
  double t_submit = 0, t_admit = 0;
  bool cancel = false;
  long long last_t = 0;   // iteration count after the last launch
  long long launches = 0; // launches the slot took part in
  int refinements = 0;    // re-solves before this one (original-LP check)
  long long iters_before = 0;
  double solve_s_before = 0;
  int tile = 0;           // tile shape candidate of its layout
  bool tile_trial = false;
};

// A bucket launch as a CUDA graph: the order copy, an event, k_batch (its
// cluster shape fixed at instantiation), an event, the state read-back and
// the completion event.  One per cluster x CTA shape; before each launch the
// copies' sizes and the kernel's grid and slot count are updated in place.
struct LaunchGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t h2d = nullptr, kern = nullptr, d2h = nullptr;
};

// one size bucket: its launch loop runs independently of the others
struct Bucket {
  Tuner tuner;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
  bool inflight = false;
  bool tail = false;       // launch used the tail shape (not timed)
  std::vector<int> order;  // slots of the launch in flight
  std::map<int, LaunchGraph> graphs;  // by cl * 4096 + block
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace gb300lp

using namespace gb300lp;

struct lp_server {
  lp_device_ctx ctx{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  cudaStream_t bs[kNumBuckets] = {nullptr, nullptr, nullptr, nullptr};
  Bucket buckets[kNumBuckets];
  int device = 0, sm_count = 0;
  long long graph_launches = 0;   // bucket launches replayed from a CUDA graph
  long long graphs_built = 0;     // bucket graphs instantiated
  long long solo_nnz = kSoloNnz;  // requests at least this large run on the single-LP path
  int solo_max = 3;               // solo requests running at once
  double launch_ms = 2.0;         // device time budget of one bucket launch
  lp_solve_opts opts{};
  unsigned char *arena = nullptr;
  size_t arena_bytes = 0;
  RangeAlloc ralloc;
  int max_slots = 0;
  SlotDesc *d_desc = nullptr;
  State *d_state = nullptr;
  int *d_order = nullptr;    // kNumBuckets x max_slots
  State *d_sout = nullptr;   // kNumBuckets x max_slots: states in launch order
  State *h_state = nullptr;  // pinned, initial states of admitted slots
  int *h_order = nullptr;    // pinned, kNumBuckets x max_slots
  State *h_sout = nullptr;   // pinned, kNumBuckets x max_slots
  std::vector<Slot> slots;
  std::deque<Request> queue;
  std::map<uint64_t, Done> done;
  std::map<uint64_t, int> where;  // ticket -> 0 queued, 1 running, 2 done
  uint64_t next_ticket = 1;
  long long n_admitted = 0, n_finished = 0, n_periods = 0, launches = 0;
  // host time spent issuing bucket launches (order copy, events, the launch,
  // the state read-back) and the device time of the completed launches
  long long host_launch_ns = 0, device_launch_ns = 0;
  size_t resident = 0, peak_resident = 0;
  std::mutex mu;
  std::mutex arena_mu;  // guards ralloc, resident, solo_blocks
  std::map<size_t, size_t> solo_blocks;
  std::vector<std::thread> solo_threads;
  int solo_running = 0;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  bool use_worker = false;
  std::string worker_err;
};

namespace {

void state_init(const lp_solve_opts &o, State &st, const Packed &pk) {
  std::memset(&st, 0, sizeof(st));
  st.rho = o.rho;
  st.beta_suff = o.beta_suff;
  st.beta_nec = o.beta_nec;
  st.beta_art = o.beta_art;
  st.theta = o.theta;
  st.eps_rel = o.eps_rel;
  st.eps_gap = o.eps_gap_rel > 0 ? o.eps_gap_rel : o.eps_rel;
  st.stop_on = 0;
  st.polish = 0;  // the cluster engine does not polish
  st.eps_infeas = o.eps_infeas;
  st.infeas_every = o.infeas_every;
  st.omega_clamp = o.primal_weight_clamp;
  st.bnorm = pk.bnorm;
  st.cnorm = pk.cnorm;
  st.off = pk.off;
  st.K = std::max(1, o.check_every);
  st.halpern = o.halpern ? 1 : 0;
  st.restarts_on = o.restarts ? 1 : 0;
  st.status = ST_SETUP;
  st.mixed_active = o.precision == LP_MIXED ? 1 : 0;
  st.stall = 0;
  st.best_rel = INFINITY;
  st.t_switch = -1;
}

// device memory of solo requests comes from the server's arena
void *arena_alloc(size_t bytes, void *user) {
  lp_server *srv = static_cast<lp_server *>(user);
  bytes = (bytes + 255) & ~size_t(255);
  std::lock_guard<std::mutex> ak(srv->arena_mu);
  size_t off = 0;
  if (!srv->ralloc.alloc(bytes, off)) return nullptr;
  srv->solo_blocks[off] = bytes;
  srv->resident += bytes;
  srv->peak_resident = std::max(srv->peak_resident, srv->resident);
  return srv->arena + off;
}

void arena_free(void *p, void *user) {
  lp_server *srv = static_cast<lp_server *>(user);
  std::lock_guard<std::mutex> ak(srv->arena_mu);
  size_t off = static_cast<unsigned char *>(p) - srv->arena;
  auto it = srv->solo_blocks.find(off);
  if (it == srv->solo_blocks.end()) return;
  srv->ralloc.release(off, it->second);
  srv->resident -= it->second;
  srv->solo_blocks.erase(it);
}

size_t largest_free(lp_server *srv) {
  std::lock_guard<std::mutex> ak(srv->arena_mu);
  size_t b = 0;
  for (auto &kv : srv->ralloc.free_) b = std::max(b, kv.second);
  return b;
}

// A large request: the single-LP grid path on its own stream, driven by its
// own host thread; device memory from the arena.  Caller holds mu.
bool start_solo(lp_server *srv, Request &rq) {
  if (srv->solo_running >= srv->solo_max) return false;
  if (largest_free(srv) < rq.solo_bytes) return false;
  srv->solo_running += 1;
  srv->where[rq.ticket] = 1;
  ++srv->n_admitted;
  const uint64_t ticket = rq.ticket;
  lp_problem *lp = rq.lp;
  const double t_submit = rq.t_submit;
  lp_solve_opts o = srv->opts;
  if (rq.eps_rel >= 0) o.eps_rel = rq.eps_rel;
  const int refinements = rq.refinements;
  const long long iters_before = rq.iters_before;
  const double solve_s_before = rq.solve_s_before;
  std::vector<double> xw = std::move(rq.xw), yw = std::move(rq.yw);
  srv->solo_threads.emplace_back([srv, ticket, lp, t_submit, o, refinements, iters_before,
                                  solve_s_before, xw = std::move(xw),
                                  yw = std::move(yw)]() mutable {
    const double t_admit = now_s();
    Done d;
    d.lp = lp;
    DeviceLP *dl = nullptr;
    // no exception may leave a thread: a failure becomes the request's
    // LP_NUMERICAL answer
    try {
      std::string err;
      int rc = LP_OK;
      cudaSetDevice(srv->device);
      lp_device_ctx ctx{};
      ctx.alloc = arena_alloc;
      ctx.free = arena_free;
      ctx.user = srv;
      ctx.stream = nullptr;
      ctx.device = srv->device;
      dl = dev_create(&ctx, err);
      if (!dl) rc = LP_ERR_CUDA;
      const HostLP &h = problem_current(lp);
      DeviceSolution sol;
      if (rc == LP_OK) rc = dev_upload(dl, h, err);
      if (!xw.empty()) o.x_init = xw.data();
      if (!yw.empty()) o.y_init = yw.data();
      if (rc == LP_OK) rc = dev_solve(dl, h, o, &d.res, sol, err);
      if (rc == LP_OK) {
        d.x = std::move(sol.x);
        d.y = std::move(sol.y);
        d.z = std::move(sol.z);
      } else {
        d.res.termination = LP_NUMERICAL;
      }
    } catch (const std::exception &) {
      d.res.termination = LP_NUMERICAL;
    }
    if (dl) dev_destroy(dl);
    const double tnow = now_s();
    d.res.t_setup_s = t_admit - t_submit;
    d.res.t_solve_s = tnow - t_admit + solve_s_before;
    d.res.t_total_s = tnow - t_submit;
    d.res.iterations += iters_before;
    d.res.refinements = refinements;
    d.res.rel_kkt_original = d.res.rel_kkt;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->done[ticket] = std::move(d);
    srv->where[ticket] = 2;
    ++srv->n_finished;
    srv->solo_running -= 1;
    srv->cv.notify_all();
  });
  return true;
}

// Admit queued requests while a slot and arena space are free (caller holds mu)
void admit(lp_server *srv) {
  while (!srv->queue.empty()) {
    Request &rq = srv->queue.front();
    if (rq.cancelled) {
      Done d;
      d.res.termination = LP_CANCELLED;
      srv->done[rq.ticket] = std::move(d);
      srv->where[rq.ticket] = 2;
      srv->queue.pop_front();
      continue;
    }
    int sid = -1;
    for (int q = 0; q < srv->max_slots; ++q)
      if (!srv->slots[q].used) {
        sid = q;
        break;
      }
    if (sid < 0) return;
    if (rq.solo) {
      if (!start_solo(srv, rq)) return;
      srv->queue.pop_front();
      continue;
    }
    size_t off = 0;
    {
      std::lock_guard<std::mutex> ak(srv->arena_mu);
      if (!srv->ralloc.alloc(rq.pk.bytes, off)) return;
      srv->resident += rq.pk.bytes;
      srv->peak_resident = std::max(srv->peak_resident, srv->resident);
    }
    Slot &sl = srv->slots[sid];
    sl = Slot();
    sl.used = true;
    sl.ticket = rq.ticket;
    sl.lp = rq.lp;
    sl.off = off;
    sl.bytes = rq.pk.bytes;
    sl.m = rq.pk.m;
    sl.n = rq.pk.n;
    sl.nnz = rq.pk.nnz;
    sl.bucket = bucket_of(rq.pk.nnz);
    sl.t_submit = rq.t_submit;
    sl.t_admit = now_s();
    sl.desc = relocate(rq.pk.rel, srv->arena + off);
    sl.rperm = std::move(rq.pk.rperm);
    sl.cperm = std::move(rq.pk.cperm);
    sl.refinements = rq.refinements;
    sl.iters_before = rq.iters_before;
    sl.tile = rq.pk.tile;
    sl.tile_trial = rq.pk.tile_trial;
    sl.solve_s_before = rq.solve_s_before;
    CK(cudaMemcpyAsync(srv->arena + off, rq.pk.blob.data(), rq.pk.blob.size(),
                       cudaMemcpyHostToDevice, srv->s));
    CK(cudaMemcpyAsync(srv->d_desc + sid, &sl.desc, sizeof(SlotDesc), cudaMemcpyHostToDevice,
                       srv->s));
    state_init(srv->opts, srv->h_state[sid], rq.pk);
    if (rq.eps_rel >= 0) srv->h_state[sid].eps_rel = srv->h_state[sid].eps_gap = rq.eps_rel;
    CK(cudaMemcpyAsync(srv->d_state + sid, &srv->h_state[sid], sizeof(State),
                       cudaMemcpyHostToDevice, srv->s));
    CK(cudaStreamSynchronize(srv->s));  // the pageable blob may be freed next
    srv->where[rq.ticket] = 1;
    ++srv->n_admitted;
    srv->queue.pop_front();
  }
}

// The shape a newly packed request gets (trial: its class is still trying).
int tile_pick(lp_server *srv, int m, long long nnz, bool &trial) {
  std::lock_guard<std::mutex> lk(g_batch_tile_mu);
  TileClass &T = g_batch_tile[tile_table_key(srv->opts.precision, m, nnz)];
  if (T.chosen >= 0) {
    trial = false;
    return T.chosen;
  }
  trial = true;
  const int c = T.next;
  T.next = (T.next + 1) % kTileCands;
  return c;
}

// A trial slot finished: its cost (ns per nonzero-iteration) for shape c.
void tile_record(lp_server *srv, int m, long long nnz, int c, double cost) {
  std::lock_guard<std::mutex> lk(g_batch_tile_mu);
  TileClass &T = g_batch_tile[tile_table_key(srv->opts.precision, m, nnz)];
  if (T.chosen >= 0) return;
  T.sum[c] += cost;
  T.cnt[c] += 1;
  for (int q = 0; q < kTileCands; ++q)
    if (T.cnt[q] < kTileSamples) return;
  int b = 0;
  for (int q = 1; q < kTileCands; ++q)
    if (T.sum[q] / T.cnt[q] < T.sum[b] / T.cnt[b]) b = q;
  T.chosen = b;
}

// Pack a batched request under its class's tile shape.
void pack_tuned(lp_server *srv, const HostLP &h, Packed &pk, const double *xw = nullptr,
                const double *yw = nullptr) {
  bool trial = false;
  const int c = tile_pick(srv, h.m, h.nnz(), trial);
  pack_request(h, pk, xw, yw, tile_shape(c));
  pk.tile = c;
  pk.tile_trial = trial;
}

BatchConst batch_const(const lp_server *srv) {
  BatchConst C;
  C.K = std::max(1, srv->opts.check_every);
  C.ruiz_iters = srv->opts.ruiz_iters;
  C.pock_chambolle = srv->opts.pock_chambolle;
  C.power_iters = srv->opts.power_iters;
  C.infeas_every = srv->opts.infeas_every;
  C.max_iter = srv->opts.max_iter;
  C.step_size = srv->opts.step_size;
  C.primal_weight = srv->opts.primal_weight;
  C.budget_ns = (long long)(srv->launch_ms * 1e6);
  return C;
}

// One bucket launch of k_batch on the bucket's stream (direct form).
void launch_bucket(lp_server *srv, int b, int nord, const Shape &sh) {
  const BatchConst C = batch_const(srv);
  const int max_clusters = std::max(1, srv->sm_count * 4 / sh.cl);
  const int nclusters = std::min(nord, max_clusters);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * sh.cl);
  cfg.blockDim = dim3(sh.block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = srv->bs[b];
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sh.cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int *d_order = srv->d_order + (size_t)b * srv->max_slots;
  State *d_sout = srv->d_sout + (size_t)b * srv->max_slots;
  if (srv->opts.precision == LP_MIXED)
    CK(cudaLaunchKernelEx(&cfg, k_batch<true>, (const SlotDesc *)srv->d_desc, srv->d_state,
                          d_order, nord, d_sout, C));
  else
    CK(cudaLaunchKernelEx(&cfg, k_batch<false>, (const SlotDesc *)srv->d_desc, srv->d_state,
                          d_order, nord, d_sout, C));
  srv->launches++;
}

// The whole bucket step (order copy, events, k_batch, state read-back) as a
// replay of the bucket's graph for this shape, instantiated on first use.
void launch_bucket_graph(lp_server *srv, int b, int nord, const Shape &sh) {
  Bucket &B = srv->buckets[b];
  BatchConst C = batch_const(srv);
  const int max_clusters = std::max(1, srv->sm_count * 4 / sh.cl);
  const int nclusters = std::min(nord, max_clusters);
  const SlotDesc *desc = srv->d_desc;
  State *dstate = srv->d_state;
  int *d_order = srv->d_order + (size_t)b * srv->max_slots;
  const int *h_order = srv->h_order + (size_t)b * srv->max_slots;
  State *d_sout = srv->d_sout + (size_t)b * srv->max_slots;
  State *h_sout = srv->h_sout + (size_t)b * srv->max_slots;
  int nord_arg = nord;
  void *args[] = {(void *)&desc, (void *)&dstate, (void *)&d_order, (void *)&nord_arg,
                  (void *)&d_sout, (void *)&C};
  cudaKernelNodeParams kp = {};
  kp.func = srv->opts.precision == LP_MIXED ? (void *)k_batch<true> : (void *)k_batch<false>;
  kp.gridDim = dim3(nclusters * sh.cl);
  kp.blockDim = dim3(sh.block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  const size_t ob = sizeof(int) * (size_t)nord, sb = sizeof(State) * (size_t)nord;
  const int key = sh.cl * 4096 + sh.block;
  auto it = B.graphs.find(key);
  if (it == B.graphs.end()) {
    LaunchGraph G;
    cudaGraphNode_t e0, e1, e2;
    CK(cudaGraphCreate(&G.g, 0));
    CK(cudaGraphAddMemcpyNode1D(&G.h2d, G.g, nullptr, 0, d_order, h_order, ob,
                                cudaMemcpyHostToDevice));
    CK(cudaGraphAddEventRecordNode(&e0, G.g, &G.h2d, 1, B.ev0));
    CK(cudaGraphAddKernelNode(&G.kern, G.g, &e0, 1, &kp));
    cudaLaunchAttributeValue v = {};
    v.clusterDim.x = sh.cl;
    v.clusterDim.y = 1;
    v.clusterDim.z = 1;
    CK(cudaGraphKernelNodeSetAttribute(G.kern, cudaLaunchAttributeClusterDimension, &v));
    CK(cudaGraphAddEventRecordNode(&e1, G.g, &G.kern, 1, B.ev1));
    CK(cudaGraphAddMemcpyNode1D(&G.d2h, G.g, &e1, 1, h_sout, d_sout, sb,
                                cudaMemcpyDeviceToHost));
    CK(cudaGraphAddEventRecordNode(&e2, G.g, &G.d2h, 1, B.ev_done));
    CK(cudaGraphInstantiate(&G.exec, G.g, 0));
    it = B.graphs.emplace(key, G).first;
    ++srv->graphs_built;
  } else {
    const LaunchGraph &G = it->second;
    CK(cudaGraphExecMemcpyNodeSetParams1D(G.exec, G.h2d, d_order, h_order, ob,
                                          cudaMemcpyHostToDevice));
    CK(cudaGraphExecKernelNodeSetParams(G.exec, G.kern, &kp));
    CK(cudaGraphExecMemcpyNodeSetParams1D(G.exec, G.d2h, h_sout, d_sout, sb,
                                          cudaMemcpyDeviceToHost));
  }
  CK(cudaGraphLaunch(it->second.exec, srv->bs[b]));
  srv->launches++;
  ++srv->graph_launches;
}

// Hand a slot's result to its ticket and free its arena block.  The slot's
// bucket has no launch in flight.  Caller holds mu.
void retire(lp_server *srv, int q, const State *S, double tnow) {
  Slot &sl = srv->slots[q];
  const bool finished = S && S->status >= 0;
  if (finished && sl.tile_trial && !sl.cancel) {
    const long long it = std::max<long long>(std::max(S->iters, S->t), 1);
    tile_record(srv, sl.m, sl.nnz, sl.tile,
                (double)S->dev_ns / ((double)std::max<long long>(sl.nnz, 1) * (double)it));
  }
  Done d;
  d.lp = sl.lp;
  d.x.assign(sl.n, 0.0);
  d.y.assign(sl.m, 0.0);
  d.z.assign(sl.n, 0.0);
  if (finished) {
    // outputs are in the slot's device order: scatter back
    std::vector<double> buf(std::max(sl.n, sl.m));
    if (sl.n) {
      CK(cudaMemcpy(buf.data(), sl.desc.xout, 8 * sl.n, cudaMemcpyDeviceToHost));
      for (int j = 0; j < sl.n; ++j) d.x[sl.cperm[j]] = buf[j];
      CK(cudaMemcpy(buf.data(), sl.desc.zout, 8 * sl.n, cudaMemcpyDeviceToHost));
      for (int j = 0; j < sl.n; ++j) d.z[sl.cperm[j]] = buf[j];
    }
    if (sl.m) {
      CK(cudaMemcpy(buf.data(), sl.desc.yout, 8 * sl.m, cudaMemcpyDeviceToHost));
      for (int i = 0; i < sl.m; ++i) d.y[sl.rperm[i]] = buf[i];
    }
  }
  lp_result &r = d.res;
  r.termination = sl.cancel ? LP_CANCELLED : (finished ? S->status : LP_TIME_LIMIT);
  if (S) {
    r.restarts = S->restarts;
    r.iterations = finished ? S->iters : S->t;
    r.rel_kkt = S->rel_kkt;
    r.rel_p = S->rel_p;
    r.rel_d = S->rel_d;
    r.rel_gap = S->rel_gap;
    r.r_p = S->r_p;
    r.r_d = S->r_d;
    r.gap = S->gap;
    r.primal_obj = S->pobj;
    r.dual_obj = S->dobj;
    r.eta = S->eta;
    r.omega = S->omega;
    r.fp32_iterations = srv->opts.precision == LP_MIXED
                            ? (S->t_switch >= 0 ? S->t_switch : r.iterations) : 0;
  }
  r.t_setup_s = sl.t_admit - sl.t_submit;  // queueing delay
  r.t_solve_s = tnow - sl.t_admit + sl.solve_s_before;
  r.t_total_s = tnow - sl.t_submit;
  r.kernel_launches = sl.launches;
  r.iterations += sl.iters_before;
  r.refinements = sl.refinements;
  r.rel_kkt_original = r.rel_kkt;
  srv->done[sl.ticket] = std::move(d);
  srv->where[sl.ticket] = 2;
  {
    std::lock_guard<std::mutex> ak(srv->arena_mu);
    srv->ralloc.release(sl.off, sl.bytes);
    srv->resident -= sl.bytes;
  }
  sl = Slot();
  ++srv->n_finished;
}

// A bucket's launch has completed: autotuner bookkeeping, then retire the
// slots that finished (or were cancelled / ran out of time).  Caller holds mu.
void complete_bucket(lp_server *srv, int b) {
  Bucket &B = srv->buckets[b];
  B.inflight = false;
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, B.ev0, B.ev1));
  srv->device_launch_ns += (long long)(ms * 1e6);
  const State *out = srv->h_sout + (size_t)b * srv->max_slots;
  const double tnow = now_s();
  double work = 0;
  for (int oi = 0; oi < (int)B.order.size(); ++oi) {
    const int q = B.order[oi];
    Slot &sl = srv->slots[q];
    const State &S = out[oi];
    work += (double)std::max<long long>(sl.nnz, 1) * (double)std::max<long long>(S.t - sl.last_t, 0);
    sl.last_t = S.t;
    sl.launches += 1;
    const bool finished = S.status >= 0;
    const bool timeout = srv->opts.time_limit_s > 0 && tnow - sl.t_admit > srv->opts.time_limit_s;
    if (finished || timeout || sl.cancel) retire(srv, q, &S, tnow);
  }
  if (work > 0 && !B.tail) B.tuner.record(1e6 * ms / work);
  B.order.clear();
}

// Start a launch for every idle bucket with live slots.  Caller holds mu.
void launch_idle(lp_server *srv) {
  for (int b = 0; b < kNumBuckets; ++b) {
    Bucket &B = srv->buckets[b];
    if (B.inflight) continue;
    // cancelled slots that never ran in this bucket's current launch
    const double tnow = now_s();
    B.order.clear();
    for (int q = 0; q < srv->max_slots; ++q) {
      Slot &sl = srv->slots[q];
      if (!sl.used || sl.bucket != b) continue;
      if (sl.cancel) {
        retire(srv, q, nullptr, tnow);
        continue;
      }
      B.order.push_back(q);
    }
    if (B.order.empty()) continue;
    // largest first (the longest slots start first)
    std::sort(B.order.begin(), B.order.end(),
              [&](int a, int c) { return srv->slots[a].nnz > srv->slots[c].nnz; });
    const int nord = (int)B.order.size();
    int *h_order = srv->h_order + (size_t)b * srv->max_slots;
    std::copy(B.order.begin(), B.order.end(), h_order);
    Shape shp = B.tuner.pick();
    // few live slots: give each the widest cluster so the tail does not run
    // on a handful of SMs (not timed for the autotuner)
    B.tail = nord * shp.cl * 4 < srv->sm_count && B.tuner.chosen >= 0;
    if (B.tail) shp = Shape{8, 256};
    cudaStream_t st = srv->bs[b];
    const auto th0 = std::chrono::steady_clock::now();
    if (srv->opts.use_graph) {
      launch_bucket_graph(srv, b, nord, shp);
    } else {
      CK(cudaMemcpyAsync(srv->d_order + (size_t)b * srv->max_slots, h_order, sizeof(int) * nord,
                         cudaMemcpyHostToDevice, st));
      CK(cudaEventRecord(B.ev0, st));
      launch_bucket(srv, b, nord, shp);
      CK(cudaEventRecord(B.ev1, st));
      CK(cudaMemcpyAsync(srv->h_sout + (size_t)b * srv->max_slots,
                         srv->d_sout + (size_t)b * srv->max_slots, sizeof(State) * nord,
                         cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(B.ev_done, st));
    }
    srv->host_launch_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(
                               std::chrono::steady_clock::now() - th0)
                               .count();
    B.inflight = true;
    ++srv->n_periods;
  }
}

// One scheduler step: admit, collect completed launches, relaunch idle
// buckets.  With `wait`, first block until some launch in flight completes.
// Returns the number of live + queued requests.  Caller holds mu.
int step(lp_server *srv, bool wait) {
  admit(srv);
  if (wait) {
    for (int b = 0; b < kNumBuckets; ++b) {
      if (srv->buckets[b].inflight) {
        CK(cudaEventSynchronize(srv->buckets[b].ev_done));
        break;
      }
    }
  }
  for (int b = 0; b < kNumBuckets; ++b) {
    Bucket &B = srv->buckets[b];
    if (!B.inflight) continue;
    cudaError_t e = cudaEventQuery(B.ev_done);
    if (e == cudaErrorNotReady) continue;
    CK(e);
    complete_bucket(srv, b);
  }
  admit(srv);
  launch_idle(srv);
  int live = (int)srv->queue.size() + srv->solo_running;
  for (int q = 0; q < srv->max_slots; ++q) live += srv->slots[q].used ? 1 : 0;
  return live;
}

bool any_inflight(const lp_server *srv) {
  for (int b = 0; b < kNumBuckets; ++b)
    if (srv->buckets[b].inflight) return true;
  return false;
}

void worker_main(lp_server *srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    int live = (int)srv->queue.size();
    for (int q = 0; q < srv->max_slots; ++q) live += srv->slots[q].used ? 1 : 0;
    if (live == 0 && !any_inflight(srv)) {
      srv->cv.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    try {
      step(srv, false);
    } catch (const std::exception &e) {
      srv->worker_err = e.what();
      srv->stop = true;
    }
    srv->cv.notify_all();
    // let submitters / pollers in while the launches run
    lk.unlock();
    std::this_thread::sleep_for(std::chrono::microseconds(20));
    lk.lock();
  }
  srv->cv.notify_all();
}

}  // namespace

extern "C" {

int lp_server_create(size_t hbm_budget_bytes, const lp_device_ctx *dev, const lp_solve_opts *opts,
                     int32_t worker, lp_server **out) {
  if (!out) {
    set_last_error("out is NULL");
    return LP_ERR_INVALID;
  }
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20)) {
    set_last_error("budget below 1 MiB");
    return LP_ERR_BUDGET;
  }
  lp_server *srv = new lp_server();
  try {
    if (dev) srv->ctx = *dev;
    srv->device = srv->ctx.device;
    lp_solve_opts_default(&srv->opts);
    if (opts) srv->opts = *opts;
    srv->opts.x_init = nullptr;
    srv->opts.y_init = nullptr;
    if (!valid_solve_opts(srv->opts) || srv->opts.polish || srv->opts.eps_gap_rel != 0.0) {
      delete srv;
      set_last_error("invalid solve options");
      return LP_ERR_INVALID;
    }
    // the budget covers the slot arena and the slot tables
    srv->max_slots = 4096;
    const size_t tables =
        srv->max_slots * (sizeof(SlotDesc) + sizeof(State) +
                          kNumBuckets * (sizeof(int) + sizeof(State))) + 4096;
    if (hbm_budget_bytes <= tables + (1u << 16)) {
      delete srv;
      set_last_error("budget too small for the slot tables");
      return LP_ERR_BUDGET;
    }
    CK(cudaSetDevice(srv->device));
    CK(cudaDeviceGetAttribute(&srv->sm_count, cudaDevAttrMultiProcessorCount, srv->device));
    if (srv->ctx.stream) {
      srv->s = static_cast<cudaStream_t>(srv->ctx.stream);
    } else {
      CK(cudaStreamCreateWithFlags(&srv->s, cudaStreamNonBlocking));
      srv->own_stream = true;
    }
    // bucket streams by size: smaller LPs get the higher scheduling priority
    // (their blocks are placed first when the buckets' launches compete for
    // SMs), larger ones a lower one; the solo lane keeps the default (lowest)
    int prio_least = 0, prio_greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    for (int b = 0; b < kNumBuckets; ++b) {
      const int prio = std::min(prio_least, prio_greatest + b);
      CK(cudaStreamCreateWithPriority(&srv->bs[b], cudaStreamNonBlocking, prio));
      Bucket &B = srv->buckets[b];
      CK(cudaEventCreate(&B.ev0));
      CK(cudaEventCreate(&B.ev1));
      CK(cudaEventCreateWithFlags(&B.ev_done, cudaEventDisableTiming));
      B.tuner.cand = candidates(b);
      B.tuner.best_ns.assign(B.tuner.cand.size(), 1e300);
    }
    srv->arena_bytes = (hbm_budget_bytes - tables) & ~size_t(255);
    void *mem = nullptr;
    if (srv->ctx.alloc) {
      mem = srv->ctx.alloc(hbm_budget_bytes, srv->ctx.user);
      if (!mem) {
        lp_server_destroy(srv);  // the streams and events made so far
        set_last_error("device allocation of the budget failed");
        return LP_ERR_OOM;
      }
    } else {
      cudaError_t e = cudaMalloc(&mem, hbm_budget_bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        lp_server_destroy(srv);
        set_last_error(std::string("device allocation of the budget failed: ") +
                       cudaGetErrorString(e));
        return LP_ERR_OOM;
      }
    }
    unsigned char *base = static_cast<unsigned char *>(mem);
    srv->arena = base;
    srv->d_desc = reinterpret_cast<SlotDesc *>(base + srv->arena_bytes);
    srv->d_state = reinterpret_cast<State *>(reinterpret_cast<unsigned char *>(srv->d_desc) +
                                             srv->max_slots * sizeof(SlotDesc));
    srv->d_sout = reinterpret_cast<State *>(reinterpret_cast<unsigned char *>(srv->d_state) +
                                            srv->max_slots * sizeof(State));
    srv->d_order = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(srv->d_sout) +
                                           kNumBuckets * srv->max_slots * sizeof(State));
    srv->ralloc.init(srv->arena_bytes);
    CK(cudaHostAlloc(reinterpret_cast<void **>(&srv->h_state), sizeof(State) * srv->max_slots,
                     cudaHostAllocDefault));
    CK(cudaHostAlloc(reinterpret_cast<void **>(&srv->h_order),
                     sizeof(int) * kNumBuckets * srv->max_slots, cudaHostAllocDefault));
    CK(cudaHostAlloc(reinterpret_cast<void **>(&srv->h_sout),
                     sizeof(State) * kNumBuckets * srv->max_slots, cudaHostAllocDefault));
    std::memset(srv->h_state, 0, sizeof(State) * srv->max_slots);
    srv->slots.assign(srv->max_slots, Slot());
    srv->use_worker = worker != 0;
    if (srv->use_worker) srv->worker = std::thread(worker_main, srv);
  } catch (const std::exception &e) {
    // whatever was made before the failure (streams, events, the arena,
    // pinned buffers) is released with the server
    const std::string msg = e.what();
    lp_server_destroy(srv);
    set_last_error(msg);
    return LP_ERR_CUDA;
  }
  *out = srv;
  return LP_OK;
}

int lp_batch_submit(lp_server *srv, lp_problem *lp, uint64_t *ticket) {
  if (!srv || !lp || !ticket) {
    set_last_error("NULL argument");
    return LP_ERR_INVALID;
  }
  try {
    const int proven = problem_proven_status(lp);
    if (proven >= 0) {
      // the presolve already decided it: done without device work
      std::lock_guard<std::mutex> lk(srv->mu);
      *ticket = srv->next_ticket++;
      Done d;
      d.res.termination = proven;
      srv->done[*ticket] = std::move(d);
      srv->where[*ticket] = 2;
      ++srv->n_admitted;
      ++srv->n_finished;
      return LP_OK;
    }
    Request rq;
    const HostLP &h = problem_current(lp);
    if (h.nnz() >= srv->solo_nnz) {
      rq.solo = true;
      rq.solo_bytes = solo_estimate(h);
      rq.pk.m = h.m;
      rq.pk.n = h.n;
      rq.pk.nnz = h.nnz();
      rq.pk.bytes = rq.solo_bytes;
    } else {
      pack_tuned(srv, h, rq.pk);
    }
    if (rq.pk.bytes > srv->arena_bytes) {
      set_last_error("request needs " + std::to_string(rq.pk.bytes) +
                     " bytes, more than the server's budget");
      return LP_ERR_BUDGET;
    }
    if (rq.pk.nnz >= (long long)INT32_MAX) {
      set_last_error("request too large (nnz >= 2^31)");
      return LP_ERR_INVALID;
    }
    rq.lp = lp;
    rq.t_submit = now_s();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (!srv->worker_err.empty()) {
      set_last_error("server worker failed: " + srv->worker_err);
      return LP_ERR_CUDA;
    }
    rq.ticket = srv->next_ticket++;
    *ticket = rq.ticket;
    srv->where[rq.ticket] = 0;
    srv->queue.push_back(std::move(rq));
    srv->cv.notify_all();
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return LP_ERR_OOM;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return LP_ERR_INVALID;
  }
  return LP_OK;
}

int lp_batch_poll(lp_server *srv, uint64_t ticket, lp_result *res, double *x, double *y) {
  if (!srv) {
    set_last_error("server is NULL");
    return LP_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  if (!srv->worker_err.empty()) {
    set_last_error("server worker failed: " + srv->worker_err);
    return LP_ERR_CUDA;
  }
  auto w = srv->where.find(ticket);
  if (w == srv->where.end()) {
    set_last_error("unknown ticket");
    return LP_ERR_INVALID;
  }
  if (w->second != 2) return LP_PENDING;
  Done &d = srv->done[ticket];
  // the original-LP check of a presolved request (postsolve + host rel-KKT,
  // O(nnz) host work) runs on this polling thread without the server lock;
  // meanwhile the ticket reads as pending
  if (d.lp && d.res.termination == LP_OPTIMAL && srv->opts.refine_original > 0) {
    Done dd = std::move(d);
    srv->done.erase(ticket);
    w->second = 3;
    lk.unlock();
    try {
      const double k = problem_original_kkt(dd.lp, dd.x.data(), dd.y.data(), dd.z.data());
      if (k >= 0) dd.res.rel_kkt_original = k;
      if (k > srv->opts.eps_rel && dd.res.refinements < srv->opts.refine_original) {
        // solve the reduced LP again ten times tighter, warm-started
        Request rq;
        rq.lp = dd.lp;
        rq.ticket = ticket;
        rq.refinements = dd.res.refinements + 1;
        rq.eps_rel = srv->opts.eps_rel * std::pow(0.1, rq.refinements);
        rq.iters_before = dd.res.iterations;
        rq.solve_s_before = dd.res.t_solve_s;
        rq.t_submit = now_s() - dd.res.t_total_s;
        const HostLP &h = problem_current(dd.lp);
        if (h.nnz() >= srv->solo_nnz) {
          rq.solo = true;
          rq.solo_bytes = solo_estimate(h);
          rq.pk.m = h.m;
          rq.pk.n = h.n;
          rq.pk.nnz = h.nnz();
          rq.pk.bytes = rq.solo_bytes;
          rq.xw = std::move(dd.x);
          rq.yw = std::move(dd.y);
        } else {
          pack_tuned(srv, h, rq.pk, dd.x.data(), dd.y.data());
        }
        lk.lock();
        // a packed re-solve also carries its warm start; if that no longer
        // fits the budget the answer stands as it is (dd is intact then)
        if (rq.pk.bytes <= srv->arena_bytes) {
          srv->where[ticket] = 0;
          srv->queue.push_back(std::move(rq));
          srv->cv.notify_all();
          return LP_PENDING;
        }
      } else {
        lk.lock();
      }
    } catch (const std::exception &e) {
      if (!lk.owns_lock()) lk.lock();
      srv->where.erase(ticket);
      set_last_error(std::string("original-LP check failed: ") + e.what());
      return LP_ERR_INVALID;
    }
    srv->done[ticket] = std::move(dd);
    w = srv->where.find(ticket);
  }
  Done &dn = srv->done[ticket];
  if (res) *res = dn.res;
  if (x && !dn.x.empty()) std::memcpy(x, dn.x.data(), 8 * dn.x.size());
  if (y && !dn.y.empty()) std::memcpy(y, dn.y.data(), 8 * dn.y.size());
  // hand the answer to the problem so lp_postsolve can map it back
  if (dn.lp && dn.res.termination >= 0 && dn.res.termination <= LP_NUMERICAL)
    problem_store_solution(dn.lp, dn.x, dn.y, dn.z);
  srv->where.erase(w);
  srv->done.erase(ticket);
  return LP_OK;
}

int lp_server_pump(lp_server *srv, int32_t periods) {
  if (!srv) {
    set_last_error("server is NULL");
    return LP_ERR_INVALID;
  }
  if (srv->use_worker) {
    set_last_error("server runs its own worker thread");
    return LP_ERR_STATE;
  }
  try {
    std::lock_guard<std::mutex> lk(srv->mu);
    CK(cudaSetDevice(srv->device));
    int live = 0;
    for (int p = 0; p < std::max(periods, 1); ++p) {
      live = step(srv, any_inflight(srv));
      if (live == 0) break;
      bool batch_live = false;
      for (const Slot &sl : srv->slots) batch_live = batch_live || sl.used;
      if (!batch_live && srv->queue.empty()) break;  // only solo requests left
    }
    return live;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return LP_ERR_CUDA;
  }
}

int lp_server_tune(lp_server *srv, int64_t solo_nnz, int32_t solo_max, double launch_ms) {
  if (!srv) {
    set_last_error("server is NULL");
    return LP_ERR_INVALID;
  }
  if (solo_max == 0 || solo_max > 64 || !(launch_ms <= 1000.0)) {
    set_last_error("solo_max must be in [1, 64] (or negative: keep) and launch_ms <= 1000");
    return LP_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (solo_nnz > 0) srv->solo_nnz = solo_nnz;
  if (solo_max >= 0) srv->solo_max = solo_max;
  if (launch_ms > 0) srv->launch_ms = launch_ms;
  return LP_OK;
}

int lp_batch_cancel(lp_server *srv, uint64_t ticket) {
  if (!srv) {
    set_last_error("server is NULL");
    return LP_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  auto w = srv->where.find(ticket);
  if (w == srv->where.end()) {
    set_last_error("unknown ticket");
    return LP_ERR_INVALID;
  }
  if (w->second == 0) {
    for (Request &rq : srv->queue)
      if (rq.ticket == ticket) rq.cancelled = true;
  } else if (w->second == 1) {
    for (Slot &sl : srv->slots)
      if (sl.used && sl.ticket == ticket) sl.cancel = true;
  }
  return LP_OK;
}

int lp_server_stats(const lp_server *srv, int64_t *out) {
  if (!srv || !out) {
    set_last_error("NULL argument");
    return LP_ERR_INVALID;
  }
  lp_server *s = const_cast<lp_server *>(srv);
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = s->n_admitted;
  out[1] = s->n_finished;
  out[2] = s->n_periods;
  out[3] = (int64_t)s->peak_resident;
  out[4] = s->launches;
  out[5] = (int64_t)s->queue.size();
  for (int b = 0; b < kNumBuckets; ++b) out[6 + b] = s->buckets[b].tuner.current();
  out[10] = s->host_launch_ns;
  out[11] = s->device_launch_ns;
  return LP_OK;
}

int lp_server_graph_stats(const lp_server *srv, int64_t *out) {
  if (!srv || !out) {
    set_last_error("NULL argument");
    return LP_ERR_INVALID;
  }
  lp_server *s = const_cast<lp_server *>(srv);
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = s->graph_launches;
  out[1] = s->graphs_built;
  return LP_OK;
}

int lp_server_tile_tuning(const lp_server *srv, double *out, int32_t cap, int32_t *nclasses) {
  if (!srv || !nclasses || cap < 0 || (cap > 0 && !out)) {
    set_last_error("lp_server_tile_tuning: invalid argument");
    return LP_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_batch_tile_mu);
  const int mixed = srv->opts.precision == LP_MIXED ? 1 : 0;
  int32_t cnt = 0;
  for (const auto &kv : g_batch_tile) cnt += (kv.first >> 20) == mixed ? 1 : 0;
  *nclasses = cnt;
  if (cnt > cap) {
    set_last_error("lp_server_tile_tuning: cap too small");
    return LP_ERR_INVALID;
  }
  double *o = out;
  for (const auto &kv : g_batch_tile) {
    if ((kv.first >> 20) != mixed) continue;
    const TileClass &T = kv.second;
    const int key = kv.first & ((1 << 20) - 1);
    o[0] = key / 64;
    o[1] = key % 64;
    o[2] = T.chosen;
    for (int c = 0; c < kTileCands; ++c) {
      o[3 + c] = T.cnt[c] > 0 ? T.sum[c] / T.cnt[c] : -1.0;
      o[3 + kTileCands + c] = T.cnt[c];
    }
    o += 3 + 2 * kTileCands;
  }
  return LP_OK;
}

void lp_server_destroy(lp_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();
  for (std::thread &t : srv->solo_threads)
    if (t.joinable()) t.join();
  cudaSetDevice(srv->device);
  cudaStreamSynchronize(srv->s);
  for (int b = 0; b < kNumBuckets; ++b) {
    if (srv->bs[b]) {
      cudaStreamSynchronize(srv->bs[b]);
      cudaStreamDestroy(srv->bs[b]);
    }
    Bucket &B = srv->buckets[b];
    for (auto &kv : B.graphs) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    B.graphs.clear();
    if (B.ev0) cudaEventDestroy(B.ev0);
    if (B.ev1) cudaEventDestroy(B.ev1);
    if (B.ev_done) cudaEventDestroy(B.ev_done);
  }
  if (srv->arena) {
    if (srv->ctx.free) srv->ctx.free(srv->arena, srv->ctx.user);
    else cudaFree(srv->arena);
  }
  if (srv->h_state) cudaFreeHost(srv->h_state);
  if (srv->h_order) cudaFreeHost(srv->h_order);
  if (srv->h_sout) cudaFreeHost(srv->h_sout);
  if (srv->own_stream) cudaStreamDestroy(srv->s);
  delete srv;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The cluster engine of lp_solve: one LP on one thread-block cluster, the
// whole solve in a few launches of the batch kernel (no per-iteration launch),
// for LPs too small to fill the GPU with the grid kernels.

namespace gb300lp {

int cluster_solve(const HostLP &h, const lp_solve_opts &o, const lp_device_ctx *ctx,
                  lp_result *res, DeviceSolution &sol, std::string &err) {
  const auto t_start = std::chrono::steady_clock::now();
  lp_device_ctx dctx{};
  if (ctx) dctx = *ctx;
  cudaStream_t s = static_cast<cudaStream_t>(dctx.stream);
  bool own_stream = false;
  unsigned char *mem = nullptr;
  auto release = [&]() {
    if (mem) {
      if (dctx.free) dctx.free(mem, dctx.user);
      else cudaFreeAsync(mem, s);
      mem = nullptr;
    }
    if (own_stream) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
      own_stream = false;
    }
  };
  try {
    CK(cudaSetDevice(dctx.device));
    if (!s) {
      CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      own_stream = true;
    }
    const int m = h.m, n = h.n;
    Packed pk;
    pack_request(h, pk);
    const bool warm = o.x_init || o.y_init;
    auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t o_desc = a256(pk.bytes);
    const size_t o_state = o_desc + a256(sizeof(SlotDesc));
    const size_t o_sout = o_state + a256(sizeof(State));
    const size_t o_order = o_sout + a256(sizeof(State));
    const size_t o_xi = o_order + 256;
    const size_t o_yi = o_xi + a256(8 * (size_t)std::max(n, 1));
    const size_t total = o_yi + a256(8 * (size_t)std::max(m, 1));
    if (dctx.alloc) {
      mem = static_cast<unsigned char *>(dctx.alloc(total, dctx.user));
      if (!mem) {
        err = "device allocation of " + std::to_string(total) + " bytes failed";
        release();
        return LP_ERR_OOM;
      }
    } else {
      cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&mem), total, s);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        mem = nullptr;
        err = "device allocation of " + std::to_string(total) + " bytes failed";
        release();
        return LP_ERR_OOM;
      }
      CK(e);
    }
    SlotDesc desc = relocate(pk.rel, mem);
    std::vector<double> xw, yw;
    if (warm) {
      // warm start in the device order (unscaled; the set-up divides by the scaling)
      xw.assign(n, 0.0);
      yw.assign(m, 0.0);
      for (int j = 0; j < n; ++j) xw[j] = o.x_init ? o.x_init[pk.cperm[j]] : 0.0;
      for (int i = 0; i < m; ++i) yw[i] = o.y_init ? o.y_init[pk.rperm[i]] : 0.0;
      desc.xinit = reinterpret_cast<const double *>(mem + o_xi);
      desc.yinit = reinterpret_cast<const double *>(mem + o_yi);
      if (n) CK(cudaMemcpyAsync(mem + o_xi, xw.data(), 8 * n, cudaMemcpyHostToDevice, s));
      if (m) CK(cudaMemcpyAsync(mem + o_yi, yw.data(), 8 * m, cudaMemcpyHostToDevice, s));
    }
    State st0;
    state_init(o, st0, pk);
    const int zero = 0;
    CK(cudaMemcpyAsync(mem, pk.blob.data(), pk.blob.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mem + o_desc, &desc, sizeof(SlotDesc), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mem + o_state, &st0, sizeof(State), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mem + o_order, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // host buffers may be freed below
    const double t_setup =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    // cluster shape by size
    const long long nnz = h.nnz();
    const int CLs = nnz < 16384 ? 1 : (nnz < 65536 ? 2 : (nnz < 262144 ? 4 : 8));
    BatchConst C;
    C.K = std::max(1, o.check_every);
    C.ruiz_iters = o.ruiz_iters;
    C.pock_chambolle = o.pock_chambolle;
    C.power_iters = o.power_iters;
    C.infeas_every = o.infeas_every;
    C.max_iter = o.max_iter;
    C.step_size = o.step_size;
    C.primal_weight = o.primal_weight;
    const double tl = o.time_limit_s > 0 ? o.time_limit_s : 1e30;
    C.budget_ns = (long long)(std::min(0.05, tl) * 1e9);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLs);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const SlotDesc *d_desc = reinterpret_cast<const SlotDesc *>(mem + o_desc);
    State *d_state = reinterpret_cast<State *>(mem + o_state);
    State *d_sout = reinterpret_cast<State *>(mem + o_sout);
    const int *d_order = reinterpret_cast<const int *>(mem + o_order);
    State hs;
    long long launches = 0;
    bool timed_out = false;
    const auto t_solve0 = std::chrono::steady_clock::now();
    for (;;) {
      if (o.precision == LP_MIXED)
        CK(cudaLaunchKernelEx(&cfg, k_batch<true>, d_desc, d_state, d_order, 1, d_sout, C));
      else
        CK(cudaLaunchKernelEx(&cfg, k_batch<false>, d_desc, d_state, d_order, 1, d_sout, C));
      ++launches;
      CK(cudaMemcpyAsync(&hs, d_sout, sizeof(State), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      trace_state("cluster", hs.t, hs.rel_kkt, hs.rel_p, hs.rel_d, hs.rel_gap, hs.omega,
                  hs.restarts, hs.mixed_active);
      if (o.verbose)
        std::fprintf(stderr, "pdhg-cluster t=%lld rel_kkt=%.3e omega=%.3e restarts=%d fp32=%d\n",
                     hs.t, hs.rel_kkt, hs.omega, hs.restarts, hs.mixed_active);
      if (hs.status >= 0) break;
      const double el =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      if (el > tl) {
        timed_out = true;
        break;
      }
    }
    const double t_solve =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_solve0).count();
    // outputs: unscale and renumber on the host
    std::vector<double> xh(n), yh(m), xc(n), yc(m), dc(n), dr(m), zz(n);
    if (n) {
      CK(cudaMemcpyAsync(xh.data(), desc.xhat, 8 * n, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(xc.data(), desc.x, 8 * n, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(dc.data(), desc.dc, 8 * n, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(zz.data(), desc.zout, 8 * n, cudaMemcpyDeviceToHost, s));
    }
    if (m) {
      CK(cudaMemcpyAsync(yh.data(), desc.yhat, 8 * m, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(yc.data(), desc.y, 8 * m, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(dr.data(), desc.dr, 8 * m, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    sol.x.assign(n, 0.0);
    sol.z.assign(n, 0.0);
    sol.xi.assign(n, 0.0);
    sol.y.assign(m, 0.0);
    sol.yi.assign(m, 0.0);
    for (int j = 0; j < n; ++j) {
      const int oj = pk.cperm[j];
      sol.x[oj] = dc[j] * xh[j];
      sol.xi[oj] = dc[j] * xc[j];
      sol.z[oj] = zz[j];
    }
    for (int i = 0; i < m; ++i) {
      const int oi = pk.rperm[i];
      sol.y[oi] = dr[i] * yh[i];
      sol.yi[oi] = dr[i] * yc[i];
    }
    sol.valid = true;
    release();
    if (res) {
      std::memset(res, 0, sizeof(*res));
      res->termination = timed_out ? LP_TIME_LIMIT : hs.status;
      res->restarts = hs.restarts;
      res->iterations = hs.status >= 0 ? hs.iters : hs.t;
      res->rel_kkt = hs.rel_kkt;
      res->rel_p = hs.rel_p;
      res->rel_d = hs.rel_d;
      res->rel_gap = hs.rel_gap;
      res->r_p = hs.r_p;
      res->r_d = hs.r_d;
      res->gap = hs.gap;
      res->primal_obj = hs.pobj;
      res->dual_obj = hs.dobj;
      res->eta = hs.eta;
      res->omega = hs.omega;
      res->t_setup_s = t_setup;
      res->t_solve_s = t_solve;
      res->t_total_s =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      res->kernel_launches = launches;
      res->fp32_iterations = o.precision == LP_MIXED
                                 ? (hs.t_switch >= 0 ? hs.t_switch : res->iterations) : 0;
    }
  } catch (const DeviceOOM &e) {
    err = e.what();
    release();
    return LP_ERR_OOM;
  } catch (const std::exception &e) {
    err = e.what();
    release();
    return LP_ERR_CUDA;
  }
  return LP_OK;
}

}  // namespace gb300lp
