// Single-LP GPU path: restarted reflected Halpern PDHG for eq. (1).
//
// Data layout in HBM (built once per problem by dev_upload):
//   * rows of A and rows of A^T (= columns of A) are each sorted by length
//     (longest first) and cut into warp tiles (see spmv_warp.cuh); the LP is
//     renumbered with those permutations, so the epilogues of the SpMV
//     kernels read and write their vectors contiguously;
//   * A (m rows) and its stored transpose A^T (n rows) in CSR with int32
//     offsets and column indices; unscaled FP64 values are kept for
//     re-solves, scaled FP64 values (and FP32 copies in mixed precision) are
//     what the iteration reads;
//   * per-row / per-column vectors in FP64.
//
// Kernels per PDHG iteration (the operator T and the Halpern step):
//   K1  g = A~^T y       fused with  xh = proj(x - tau (c~ - g)), xbar = 2 xh - x,
//                                     x <- lam((1+rho) xh - rho x) + (1-lam) x0
//   K2  h = A~ xbar      fused with  v = y - sigma h, yh = v + sigma proj(-v / sigma),
//                                     y <- lam((1+rho) yh - rho y) + (1-lam) y0
// and every K-th iteration (the check):
//   K1/K2 also write xh, yh and block partials of ||x - xh||^2, ||xh - x0||^2, ...
//   K3a h = A~ xh        fused with  primal residual and the y part of the dual objective
//   K3b g = A~^T yh      fused with  dual residual, lambda part of the dual objective, c^T x
//   K4  one CTA: fixed-order reduction of the partials, rel-KKT, termination,
//       restart test and primal-weight update (device state, no host round trip)
//   K5  on restart: x = x0 = xh, y = y0 = yh
// A CUDA graph holds one check iteration plus K - 1 plain iterations and the
// D2H copy of the state word; the host replays it until the state says done.
//
// FP64 instruction budget (GB300 runs FP64 at about 2 lanes per clock per
// SM): the SpMV costs one DFMA per nonzero at full lanes; the epilogues use
// precomputed Halpern coefficients a = lam (1 + rho), b = -lam rho,
// g = 1 - lam and the division-free dual prox v + clamp(-v, sigma l, sigma u).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "device_common.cuh"
#include "lp_internal.h"
#include "pdhg_state.cuh"
#include "host_parallel.h"
#include "layout.h"
#include "pdhg_epi.cuh"
#include "spmv_warp.cuh"

namespace gb300lp {

#ifndef GB300_BLOCK
#define GB300_BLOCK 256
#endif
constexpr int kBlock = GB300_BLOCK;
#ifndef GB300_MIN_BLOCKS
#define GB300_MIN_BLOCKS (1024 / GB300_BLOCK)
#endif
constexpr int kMinBlocks = GB300_MIN_BLOCKS;
// Resident CTAs per SM of the iteration kernels K1 / K2: the FP64 ones run
// three (80 registers, no spills), the mixed ones kMinBlocks (64 registers);
// a solve's grid follows its precision.
#ifndef GB300_MIN_BLOCKS_FP64
#define GB300_MIN_BLOCKS_FP64 3
#endif
template <typename T>
struct IterBlocks {
  static constexpr int value = sizeof(T) == 8 ? GB300_MIN_BLOCKS_FP64 : kMinBlocks;
};

// deterministic block reduction of NQL accumulators into partials[q * GP + block]
// (GP: the stride of a quantity, the grid's G slots followed by one slot per
// segmented row)
template <int NQL>
__device__ __forceinline__ void store_partials(double (&acc)[NQL], const int (&qidx)[NQL],
                                               double *partials, int GP) {
  __shared__ double sh[NQL][kBlock / 32];
#pragma unroll
  for (int q = 0; q < NQL; ++q) {
    double v = warp_sum(acc[q]);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQL) {
    double s = 0;
    for (int w = 0; w < kBlock / 32; ++w) s += sh[threadIdx.x][w];
    partials[qidx[threadIdx.x] * GP + blockIdx.x] = s;
  }
}

// fixed-order sum of one quantity's GP partials by a whole CTA; result in all threads
__device__ double reduce_partials(const double *partials, int q, int GP) {
  __shared__ double sh[kBlock / 32];
  __shared__ double out;
  double s = 0;
  for (int b = threadIdx.x; b < GP; b += blockDim.x) s += partials[q * GP + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
    out = t;
  }
  __syncthreads();
  double r = out;
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// scaling (Ruiz passes, then Pock-Chambolle alpha = 1)

// d_new[r] = d_self[r] / sqrt(max or sum over the row of |scaled a|), where the
// scaled entry is (dr_i |a_ij|) dc_j; for rows of A^T (TRANSPOSED) the row
// scale is dc and the other one dr.
template <bool TRANSPOSED, bool SUM>
__global__ void k_scale_pass(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ a0, const double *__restrict__ dself,
                             const double *__restrict__ dother, double *__restrict__ dnew) {
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += warps) {
    double acc = 0.0;
    const double ds = dself[r];
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      double v = TRANSPOSED ? (dother[ci[k]] * fabs(a0[k])) * ds : (ds * fabs(a0[k])) * dother[ci[k]];
      acc = SUM ? acc + v : fmax(acc, v);
    }
    acc = SUM ? warp_sum(acc) : warp_max(acc);
    if (lane == 0) dnew[r] = acc > 0.0 ? ds / sqrt(acc) : ds;
  }
}

// scaled values (dr_i a_ij) dc_j in FP64 and optionally FP32
template <bool TRANSPOSED>
__global__ void k_apply_matrix(int rows, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double *__restrict__ a0, const double *__restrict__ dself,
                               const double *__restrict__ dother, double *__restrict__ out,
                               float *__restrict__ outf) {
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += warps) {
    const double ds = dself[r];
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) {
      double v = TRANSPOSED ? (dother[ci[k]] * a0[k]) * ds : (ds * a0[k]) * dother[ci[k]];
      out[k] = v;
      if (outf) outf[k] = (float)v;
    }
  }
}

// c~ = dc c, lx~ = lx / dc, ux~ = ux / dc; partial ||c~||^2
__global__ void k_apply_cols(int n, const double *__restrict__ c0, const double *__restrict__ lx0,
                             const double *__restrict__ ux0, const double *__restrict__ dc,
                             double *__restrict__ c, double *__restrict__ lx,
                             double *__restrict__ ux, double *partials, int GP) {
  double acc[1] = {0.0};
  const int qi[1] = {Q_CN};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double d = dc[j];
    double cj = d * c0[j];
    c[j] = cj;
    lx[j] = lx0[j] / d;
    ux[j] = ux0[j] / d;
    acc[0] += cj * cj;
  }
  store_partials<1>(acc, qi, partials, GP);
}

// lc~ = dr lc, uc~ = dr uc; partial ||bhat~||^2 (finite sides, equality once)
__global__ void k_apply_rows(int m, const double *__restrict__ lc0, const double *__restrict__ uc0,
                             const double *__restrict__ dr, double *__restrict__ lc,
                             double *__restrict__ uc, double *partials, int GP) {
  double acc[1] = {0.0};
  const int qi[1] = {Q_BN};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double d = dr[i];
    double l = d * lc0[i], u = d * uc0[i];
    lc[i] = l;
    uc[i] = u;
    bool lf = isfinite(l), uf = isfinite(u);
    if (lf) acc[0] += l * l;
    if (uf && !(lf && l == u)) acc[0] += u * u;
  }
  store_partials<1>(acc, qi, partials, GP);
}

__global__ void k_fill(double *p, double v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------------------------
// SpMV kernels: every SpMV below walks the warp-tile table of its matrix with
// the engine of spmv_warp.cuh (one warp per tile, no CTA barrier).

struct MatDev {
  const int2 *tiles;
  int ntiles;
  int nlong;  // rows [0, nlong) are long rows reduced by a whole CTA
  const int *rp, *ci;
  SegCtx seg;  // segmented rows (sink: the partials of the launching kernel)
};

// the matrix with its segment sums' per-row slots in `partials` (stride GP,
// after the G per-CTA slots)
__host__ __device__ __forceinline__ SegCtx seg_sink(SegCtx s, double *partials, int GP, int G) {
  s.sink = AccSink{partials, GP, G};
  return s;
}

// kBlock / 32 accumulators of shared memory for the whole-CTA rows
template <typename T, typename V, typename Acc>
__device__ __forceinline__ Acc *red_smem() {
  __shared__ Acc red[kBlock / 32];
  return red;
}

__global__ void __launch_bounds__(kBlock, kMinBlocks) k_spmv_store(MatDev M, const double *__restrict__ va,
                                                       const double *__restrict__ vec, double *out) {
  StoreSqEpi<double> e{out, 0.0};
  SegCtx sc = M.seg;
  sc.sink = AccSink{nullptr, 0, 0};
  warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, vec, e,
                                    red_smem<double, double, double>(), blockIdx.x, gridDim.x,
                                    sc);
}

// QI: Q_PW for the A^T passes, Q_PWA for the final pass over A
template <int QI>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_spmv_store_sq(MatDev M, const double *__restrict__ va,
                                                          const double *__restrict__ vec,
                                                          double *out, double *partials, int GP) {
  StoreSqEpi<double, QI> e{out, 0.0};
  warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, vec, e,
                                    red_smem<double, double, double>(), blockIdx.x, gridDim.x,
                                    seg_sink(M.seg, partials, GP, gridDim.x));
  double acc[1] = {e.acc};
  const int qi[1] = {QI};
  store_partials<1>(acc, qi, partials, GP);
}

// v = w / ||w|| (every CTA reduces the partials in the same fixed order); a
// zero w (the start was orthogonal to A's row space) continues from the
// fallback start vector
__global__ void k_normalize(int n, const double *__restrict__ w, double *__restrict__ v,
                            const double *__restrict__ fallback, const double *partials, int GP) {
  double nw = sqrt(reduce_partials(partials, Q_PW, GP));
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    v[j] = nw > 0.0 ? w[j] / nw : fallback[j];
}

// ---------------------------------------------------------------------------
// state set-up

__global__ void k_setup_final(State *st, const double *partials, int GP, double eta_given,
                              double omega_given, int power_done) {
  double cn = sqrt(reduce_partials(partials, Q_CN, GP));
  double bn = sqrt(reduce_partials(partials, Q_BN, GP));
  double pw = power_done ? sqrt(reduce_partials(partials, Q_PWA, GP)) : 0.0;
  if (threadIdx.x == 0) {
    double eta = eta_given > 0 ? eta_given : (pw > 0 ? 0.998 / pw : 1.0);
    double om = omega_given > 0 ? omega_given : ((cn > 0 && bn > 0) ? cn / bn : 1.0);
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
    st->status = ST_RUNNING;
    st->restart_flag = 0;
    st->r0 = st->r_prev = st->last_r = 0.0;
    st->rel_kkt = INFINITY;
  }
}

__global__ void k_init_x(int n, const double *__restrict__ lx, const double *__restrict__ ux,
                         const double *__restrict__ dc, const double *__restrict__ xinit,
                         double *x, double *x0) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double v = xinit ? xinit[j] / dc[j] : clampd(0.0, lx[j], ux[j]);
    x[j] = v;
    x0[j] = v;
  }
}

__global__ void k_init_y(int m, const double *__restrict__ dr, const double *__restrict__ yinit,
                         double *y, double *y0, float2 *yf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double v = yinit ? yinit[i] / dr[i] : 0.0;
    y[i] = v;
    y0[i] = v;
    if (yf) yf[i] = split_f2(v);
  }
}

// 1 / dr and 1 / dc for the unscaling in the KKT kernels
__global__ void k_reciprocal(int n, const double *__restrict__ d, double *__restrict__ inv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    inv[i] = 1.0 / d[i];
}

// ---------------------------------------------------------------------------
// the iteration kernels

// T = float: the mixed-precision kernel; while st->mixed_active is set it
// multiplies the FP32 values by the float pairs of the gathered vector with
// compensated sums, after the switch it runs the FP64 SpMV (va64, y)
template <typename T, bool CHECK>
__global__ void __launch_bounds__(kBlock, IterBlocks<T>::value) k_primal(
    MatDev M, const T *__restrict__ va, const double *__restrict__ va64,
    const double *__restrict__ y, const float2 *__restrict__ yf, const double *__restrict__ c,
    const double *__restrict__ lx, const double *__restrict__ ux, double *x, double *x0,
    double *xbar, float2 *xbar_f, double *xhat, const State *__restrict__ st, int j,
    double *partials, int GP) {
  if (st->status != ST_RUNNING) return;
  constexpr bool MIXED = sizeof(T) == 4;
  double acc[2];
  const SegCtx sc = seg_sink(M.seg, CHECK ? partials : nullptr, GP, gridDim.x);
  if (MIXED && st->mixed_active) {
    PrimalEpi<CHECK, true> e{c, lx, ux, x, x0, xbar, xhat, xbar_f, st->tau,
                             halpern_coeffs(st, j), 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    warp_spmv<T, float2, F2>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, yf, e,
                             red_smem<T, float2, F2>(), blockIdx.x, gridDim.x, sc);
    acc[0] = e.acc0;
    acc[1] = e.acc1;
  } else {
    PrimalEpi<CHECK, false> e{c, lx, ux, x, x0, xbar, xhat, xbar_f, st->tau,
                              halpern_coeffs(st, j), 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va64, y, e,
                                      red_smem<double, double, double>(), blockIdx.x,
                                      gridDim.x, sc);
    acc[0] = e.acc0;
    acc[1] = e.acc1;
  }
  if (CHECK) {
    const int qi[2] = {Q_XRES, Q_XD};
    store_partials<2>(acc, qi, partials, GP);
  }
}

template <typename T, bool CHECK>
__global__ void __launch_bounds__(kBlock, IterBlocks<T>::value) k_dual(
    MatDev M, const T *__restrict__ va, const double *__restrict__ va64,
    const double *__restrict__ xbar, const float2 *__restrict__ xbar_f,
    const double *__restrict__ lc, const double *__restrict__ uc, double *y, double *y0,
    float2 *yf, double *yhat, const State *__restrict__ st, int j, double *partials, int GP) {
  if (st->status != ST_RUNNING) return;
  constexpr bool MIXED = sizeof(T) == 4;
  double acc[2];
  const SegCtx sc = seg_sink(M.seg, CHECK ? partials : nullptr, GP, gridDim.x);
  if (MIXED && st->mixed_active) {
    DualEpi<CHECK, true> e{lc, uc, y, y0, yhat, yf, st->sigma, halpern_coeffs(st, j), 0.0, 0.0,
                           0.0, 0.0, 0.0, 0.0};
    warp_spmv<T, float2, F2>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, xbar_f, e,
                             red_smem<T, float2, F2>(), blockIdx.x, gridDim.x, sc);
    acc[0] = e.acc0;
    acc[1] = e.acc1;
  } else {
    DualEpi<CHECK, false> e{lc, uc, y, y0, yhat, yf, st->sigma, halpern_coeffs(st, j), 0.0, 0.0,
                            0.0, 0.0, 0.0, 0.0};
    warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va64, xbar, e,
                                      red_smem<double, double, double>(), blockIdx.x,
                                      gridDim.x, sc);
    acc[0] = e.acc0;
    acc[1] = e.acc1;
  }
  if (CHECK) {
    const int qi[2] = {Q_YRES, Q_YD};
    store_partials<2>(acc, qi, partials, GP);
  }
}

__global__ void __launch_bounds__(kBlock, kMinBlocks) k_kkt_rows(
    MatDev M, const double *__restrict__ va, const double *__restrict__ xhat,
    const double *__restrict__ dr, const double *__restrict__ idr,
    const double *__restrict__ lc0, const double *__restrict__ uc0,
    const double *__restrict__ yhat, const State *__restrict__ st, int force, double *partials,
    int GP) {
  if (!force && st->status != ST_RUNNING) return;
  KktRowEpi e{dr, idr, lc0, uc0, yhat, 0.0, 0.0, 0.0};
  warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, xhat, e,
                                    red_smem<double, double, double>(), blockIdx.x, gridDim.x,
                                    seg_sink(M.seg, partials, GP, gridDim.x));
  double acc[3] = {e.rp2, e.rdy2, e.dy};
  const int qi[3] = {Q_RP, Q_RDY, Q_DY};
  store_partials<3>(acc, qi, partials, GP);
}

__global__ void __launch_bounds__(kBlock, kMinBlocks) k_kkt_cols(
    MatDev M, const double *__restrict__ va, const double *__restrict__ yhat,
    const double *__restrict__ c, const double *__restrict__ dc, const double *__restrict__ idc,
    const double *__restrict__ c0, const double *__restrict__ lx0, const double *__restrict__ ux0,
    const double *__restrict__ xhat, double *zbuf, const State *__restrict__ st, int force,
    double *partials, int GP) {
  if (!force && st->status != ST_RUNNING) return;
  KktColEpi e{c, dc, idc, c0, lx0, ux0, xhat, zbuf, 0.0, 0.0, 0.0};
  warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, yhat, e,
                                    red_smem<double, double, double>(), blockIdx.x, gridDim.x,
                                    seg_sink(M.seg, partials, GP, gridDim.x));
  double acc[3] = {e.rd2, e.dl, e.p};
  const int qi[3] = {Q_RD, Q_DL, Q_P};
  store_partials<3>(acc, qi, partials, GP);
}

// Infeasibility test of a check (skipped unless due): the direction
// (xh - x0, yh - y0); K_I0 the columns (c^T d, cone violation of d; d~ into
// dbuf), K_I1 the rows of A at d~ (cone violation of A d; projected w~ into
// wbuf, dual-ray objective), K_I2 the rows of A^T at w~ (residual, objective)
__global__ void k_inf_prep(const State *__restrict__ st, int n, const double *__restrict__ xhat,
                           const double *__restrict__ x0, const double *__restrict__ dc,
                           const double *__restrict__ c0, const double *__restrict__ lx0,
                           const double *__restrict__ ux0, double *dbuf, double *partials,
                           int GP) {
  if (st->status != ST_RUNNING || !infeas_due(st->t, st->K, st->infeas_every)) return;
  double acc[2] = {0.0, 0.0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    inf_col_prep(j, xhat, x0, dc, c0, lx0, ux0, dbuf, acc[0], acc[1]);
  const int qi[2] = {Q_ICD, Q_IPVC};
  store_partials<2>(acc, qi, partials, GP);
}

__global__ void __launch_bounds__(kBlock, kMinBlocks) k_inf_rows(
    MatDev M, const double *__restrict__ va, const double *__restrict__ dbuf,
    const double *__restrict__ dr, const double *__restrict__ idr,
    const double *__restrict__ lc0, const double *__restrict__ uc0,
    const double *__restrict__ yhat, const double *__restrict__ y0, double *wbuf,
    const State *__restrict__ st, double *partials, int GP) {
  if (st->status != ST_RUNNING || !infeas_due(st->t, st->K, st->infeas_every)) return;
  InfRowEpi e{dr, idr, lc0, uc0, yhat, y0, wbuf, 0.0, 0.0};
  warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, dbuf, e,
                                    red_smem<double, double, double>(), blockIdx.x, gridDim.x,
                                    seg_sink(M.seg, partials, GP, gridDim.x));
  double acc[2] = {e.v2, e.dobj};
  const int qi[2] = {Q_IPVR, Q_IDOR};
  store_partials<2>(acc, qi, partials, GP);
}

__global__ void __launch_bounds__(kBlock, kMinBlocks) k_inf_cols(
    MatDev M, const double *__restrict__ va, const double *__restrict__ wbuf,
    const double *__restrict__ idc, const double *__restrict__ lx0,
    const double *__restrict__ ux0, const State *__restrict__ st, double *partials, int GP) {
  if (st->status != ST_RUNNING || !infeas_due(st->t, st->K, st->infeas_every)) return;
  InfColEpi e{idc, lx0, ux0, 0.0, 0.0};
  warp_spmv<double, double, double>(M.nlong, M.tiles, M.ntiles, M.rp, M.ci, va, wbuf, e,
                                    red_smem<double, double, double>(), blockIdx.x, gridDim.x,
                                    seg_sink(M.seg, partials, GP, gridDim.x));
  double acc[2] = {e.r2, e.dobj};
  const int qi[2] = {Q_IDR, Q_IDOC};
  store_partials<2>(acc, qi, partials, GP);
}

// K4: the check.  eval_only: fill in the KKT fields and mark ITER_LIMIT.
// One warp per quantity (fixed lane stride over the G partials, fixed
// shuffle tree: deterministic), all quantities' loads in flight at once; the
// infeasibility quantities only on the checks that test for it.
__global__ void k_check(State *st, const double *partials, int GP, int eval_only) {
  if (!eval_only && st->status != ST_RUNNING) return;
  __shared__ double q[NQ];
  const int nq = (!eval_only && infeas_due(st->t, st->K, st->infeas_every)) ? Q_CN : Q_ICD;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < nq; i += nw) {
    double s = 0.0;
    for (int b = lane; b < GP; b += 32) s += partials[i * GP + b];
    s = warp_sum(s);
    if (lane == 0) q[i] = s;
  }
  for (int i = nq + (int)threadIdx.x; i < NQ; i += blockDim.x) q[i] = 0.0;
  __syncthreads();
  if (threadIdx.x != 0) return;
  check_update(st, q, eval_only != 0);
}

// Feasibility polishing (State::polish; the phases run on the host's
// orders with the iteration kernels): resume the check that asked for it
// after a failed attempt -- its quantities are in st->pq -- with the next
// attempt allowed at 2t.
__global__ void k_check_resume(State *st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->status = ST_RUNNING;
  st->next_polish = 2 * st->t;
  double q[NQ];
  for (int i = 0; i < NQ; ++i) q[i] = st->pq[i];
  check_update(st, q, false);
}

// the dual phase's problem: every finite entry of v set to 0
__global__ void k_zero_finite(int n, double *v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (isfinite(v[i])) v[i] = 0.0;
}

// a phase's start (scaled): x = x0 = xs, y = y0 = ys (0 where NULL); yf the
// float pairs of y when given
__global__ void k_set_point(int n, int m, const double *__restrict__ xs,
                            const double *__restrict__ ys, double *x, double *x0, double *y,
                            double *y0, float2 *yf) {
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int j = i0; j < n; j += st) {
    const double v = xs ? xs[j] : 0.0;
    x[j] = v;
    x0[j] = v;
  }
  for (int i = i0; i < m; i += st) {
    const double v = ys ? ys[i] : 0.0;
    y[i] = v;
    y0[i] = v;
    if (yf) yf[i] = split_f2(v);
  }
}

// yf = the float pairs of y (after y is restored)
__global__ void k_split_y(int m, const double *__restrict__ y, float2 *yf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    yf[i] = split_f2(y[i]);
}

// K5: on restart, x = x0 = xh and y = y0 = yh
__global__ void k_restart(const State *__restrict__ st, int n, int m, double *x, double *x0,
                          const double *__restrict__ xhat, double *y, double *y0,
                          const double *__restrict__ yhat, float2 *yf) {
  if (st->status != ST_RUNNING || !st->restart_flag) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double v = xhat[j];
    x[j] = v;
    x0[j] = v;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double v = yhat[i];
    y[i] = v;
    y0[i] = v;
    if (yf) yf[i] = split_f2(v);
  }
}

// unscaled outputs in the permuted order
__global__ void k_unscale(int n, int m, const double *__restrict__ dc, const double *__restrict__ dr,
                          const double *__restrict__ xhat, const double *__restrict__ yhat,
                          const double *__restrict__ x, const double *__restrict__ y,
                          double *out_xh, double *out_yh, double *out_x, double *out_y) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    out_xh[j] = dc[j] * xhat[j];
    out_x[j] = dc[j] * x[j];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    out_yh[i] = dr[i] * yhat[i];
    out_y[i] = dr[i] * y[i];
  }
}

// ---------------------------------------------------------------------------
// host side

constexpr size_t kSmem64 = 0;  // the warp engine needs no dynamic shared memory

// CUDA events owned by a scope: destroyed when it ends, also when a CUDA
// error (an exception from CK) or an early return leaves it
struct ScopedEvents {
  std::vector<cudaEvent_t> ev;
  ScopedEvents() = default;
  ScopedEvents(const ScopedEvents &) = delete;
  ScopedEvents &operator=(const ScopedEvents &) = delete;
  ~ScopedEvents() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  cudaEvent_t make(unsigned flags = cudaEventDefault) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, flags));
    ev.push_back(e);
    return e;
  }
};
constexpr size_t kSmem32 = 0;
constexpr int kDefaultShape = 3;  // tile_candidates()[3]: run_max 16, 2048 nonzeros

struct DeviceLP {
  lp_device_ctx ctx{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int device = 0;
  int sm_count = 0;
  bool uploaded = false;
  int m = 0, n = 0;
  long long nnz = 0;
  std::vector<int> rperm, cperm;  // new -> old
  int ntilesA = 0, ntilesT = 0, nlongA = 0, nlongT = 0;
  int2 *tilesA = nullptr, *tilesT = nullptr;
  // segmented rows of A and A^T (see spmv_warp.cuh)
  int *segbaseA = nullptr, *segbaseT = nullptr, *segcntA = nullptr, *segcntT = nullptr;
  double *segpartA = nullptr, *segpartT = nullptr;
  int seglenA = 0, seglenT = 0, nsegrowsA = 0, nsegrowsT = 0;
  // every candidate shape's tile table (host), and which one is on the device
  std::vector<TilePlan> plansA, plansT;
  int planA = -1, planT = -1;
  int G = 1;   // CTAs of the grid-wide kernels of the current solve
  int G64 = 1, G32 = 1;  // ... of an FP64 / a mixed solve
  int GP = 1;  // stride of a quantity in `partials`: G + the most segmented rows
  int *A_rp = nullptr, *A_ci = nullptr, *T_rp = nullptr, *T_ci = nullptr;
  double *A_v0 = nullptr, *T_v0 = nullptr, *A_v = nullptr, *T_v = nullptr;
  float *A_vf = nullptr, *T_vf = nullptr;
  double *c0 = nullptr, *lx0 = nullptr, *ux0 = nullptr, *lc0 = nullptr, *uc0 = nullptr;
  double *c = nullptr, *lx = nullptr, *ux = nullptr, *lc = nullptr, *uc = nullptr;
  double *dr = nullptr, *dc = nullptr, *dr2 = nullptr, *dc2 = nullptr;
  double *dr_main = nullptr, *dc_main = nullptr;  // where dr / dc live after scaling
  double *idr = nullptr, *idc = nullptr;
  double *x = nullptr, *x0 = nullptr, *xbar = nullptr, *xhat = nullptr;
  double *y = nullptr, *y0 = nullptr, *yhat = nullptr, *zbuf = nullptr;
  double *pv = nullptr, *pv0 = nullptr, *pw = nullptr, *pu = nullptr;
  // feasibility polishing: the main iterate, anchor and T(z) kept while the
  // phases run, and the primal phase's x (allocated on first use)
  double *bx = nullptr, *bx0 = nullptr, *bxh = nullptr, *bxp = nullptr;
  double *by = nullptr, *by0 = nullptr, *byh = nullptr;
  int infeas_every = 0;  // of the current solve (host copy of the state's)
  // last tile-shape measurement: mean ms of K1 (rows of A^T) and K2 (rows of
  // A) per candidate, or empty when the choice came from the cache / opts
  std::vector<double> tune_msT, tune_msA;
  double *ox = nullptr, *oy = nullptr, *oxi = nullptr, *oyi = nullptr;
  float2 *xbar_f = nullptr, *yf = nullptr;  // mixed: x-bar and y as float pairs
  double *partials = nullptr;
  State *st = nullptr;
  State *hst = nullptr;
  double *hbuf = nullptr;  // pinned staging for warm starts
  double bnorm = 0, cnorm = 0, off = 0;
  std::vector<void *> allocs;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_K[2] = {0, 0};
  int graph_inf[2] = {0, 0};  // whether the graph holds the infeasibility test
  long long launches = 0;
  int last_precision = -1;
  void *flush = nullptr;
  size_t flush_bytes = 0;

  MatDev matA() const {
    return MatDev{tilesA, ntilesA, nlongA, A_rp, A_ci,
                  SegCtx{segbaseA, segpartA, segcntA, seglenA, AccSink{nullptr, 0, 0}}};
  }
  MatDev matT() const {
    return MatDev{tilesT, ntilesT, nlongT, T_rp, T_ci,
                  SegCtx{segbaseT, segpartT, segcntT, seglenT, AccSink{nullptr, 0, 0}}};
  }

  void *dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (ctx.alloc) {
      p = ctx.alloc(bytes, ctx.user);
      if (!p) throw DeviceOOM("device allocation of " + std::to_string(bytes) + " bytes failed");
    } else {
      cudaError_t e = cudaMallocAsync(&p, bytes, s);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        throw DeviceOOM("device allocation of " + std::to_string(bytes) + " bytes failed");
      }
      CK(e);
    }
    allocs.push_back(p);
    return p;
  }
  template <typename T>
  T *dalloc_n(size_t n) {
    return static_cast<T *>(dalloc(n * sizeof(T)));
  }
  void release_all() {
    for (int q = 0; q < 2; ++q)
      if (graph[q]) {
        cudaGraphExecDestroy(graph[q]);
        graph[q] = nullptr;
      }
    for (void *p : allocs) {
      if (ctx.free) ctx.free(p, ctx.user);
      else cudaFreeAsync(p, s);
    }
    allocs.clear();
    flush = nullptr;
    bx = bx0 = bxh = bxp = by = by0 = byh = nullptr;
    uploaded = false;
  }
  // persistent grid for a warp-tile table (8 warps per CTA), at most G CTAs
  int grid_tiles(int ntiles, int nlong) const {
    return std::max(1, std::min(std::max((ntiles + kBlock / 32 - 1) / (kBlock / 32), nlong), G));
  }
  int grid_for(long long work) const {
    long long g = (work + kBlock - 1) / kBlock;
    g = std::max<long long>(1, std::min<long long>(g, (long long)sm_count * 8));
    return (int)g;
  }
};

// Tile shapes of the single-LP path (segmented long rows): run_max 8, 16, 32,
// 64 entries per lane (segments of 32 run_max entries), times 512 or 2048
// nonzeros per tile.
const std::vector<TileShape> &tile_candidates() {
  static const std::vector<TileShape> c = [] {
    std::vector<TileShape> v;
    for (int r : {8, 16, 32, 64})
      for (int t : {512, 2048}) v.push_back(TileShape{r, t, true});
    return v;
  }();
  return c;
}

// index of a candidate shape, or -1
int tile_candidate_index(int run_max, int tile_nnz) {
  const std::vector<TileShape> &c = tile_candidates();
  for (size_t i = 0; i < c.size(); ++i)
    if (c[i].run_max == run_max && c[i].tile_nnz == tile_nnz) return (int)i;
  return -1;
}

// Put candidate plans ca (rows of A) and ct (rows of A^T) on the device,
// in stream order on the library stream.  A change drops the captured
// iteration graphs (their kernel arguments hold the tile counts).
void install_plan(DeviceLP *d, int ca, int ct) {
  if (ca == d->planA && ct == d->planT) return;
  auto put = [d](const TilePlan &p, int2 *tiles, int *segbase, int &ntiles, int &nlong,
                 int &nsegrows, int &seglen) {
    ntiles = (int)p.tiles.size();
    nlong = p.nlong;
    nsegrows = p.nsegrows;
    seglen = p.seg_len;
    if (ntiles)
      CK(cudaMemcpyAsync(tiles, p.tiles.data(), sizeof(int2) * ntiles, cudaMemcpyHostToDevice,
                         d->s));
    CK(cudaMemcpyAsync(segbase, p.seg_base.data(), sizeof(int) * p.seg_base.size(),
                       cudaMemcpyHostToDevice, d->s));
  };
  put(d->plansA[ca], d->tilesA, d->segbaseA, d->ntilesA, d->nlongA, d->nsegrowsA, d->seglenA);
  put(d->plansT[ct], d->tilesT, d->segbaseT, d->ntilesT, d->nlongT, d->nsegrowsT, d->seglenT);
  d->planA = ca;
  d->planT = ct;
  // the per-row slots of segmented rows (after the G per-CTA slots of every
  // quantity) are summed by every reduction: drop what the previous plan's
  // segmented rows left there
  if (d->GP > d->G)
    for (int q = 0; q < NQ; ++q)
      CK(cudaMemsetAsync(d->partials + (size_t)q * d->GP + d->G, 0,
                         sizeof(double) * (d->GP - d->G), d->s));
  for (int q = 0; q < 2; ++q)
    if (d->graph[q]) {
      CK(cudaGraphExecDestroy(d->graph[q]));
      d->graph[q] = nullptr;
    }
}

DeviceLP *dev_create(const lp_device_ctx *ctx, std::string &err) {
  DeviceLP *d = new DeviceLP();
  try {
    if (ctx) d->ctx = *ctx;
    d->device = d->ctx.device;
    CK(cudaSetDevice(d->device));
    CK(cudaDeviceGetAttribute(&d->sm_count, cudaDevAttrMultiProcessorCount, d->device));
    if (d->ctx.stream) {
      d->s = static_cast<cudaStream_t>(d->ctx.stream);
    } else {
      CK(cudaStreamCreateWithFlags(&d->s, cudaStreamNonBlocking));
      d->own_stream = true;
    }
    CK(cudaHostAlloc(reinterpret_cast<void **>(&d->hst), sizeof(State), cudaHostAllocDefault));
  } catch (const std::exception &e) {
    err = e.what();
    dev_destroy(d);  // also the stream made before the failure
    return nullptr;
  }
  return d;
}

bool dev_uploaded(const DeviceLP *d) { return d && d->uploaded; }

void dev_destroy(DeviceLP *d) {
  if (!d) return;
  cudaSetDevice(d->device);
  d->release_all();
  cudaStreamSynchronize(d->s);
  if (d->hst) cudaFreeHost(d->hst);
  if (d->hbuf) cudaFreeHost(d->hbuf);
  if (d->own_stream) cudaStreamDestroy(d->s);
  delete d;
}

int dev_upload(DeviceLP *d, const HostLP &h, std::string &err) {
  try {
    CK(cudaSetDevice(d->device));
    d->release_all();
    if (h.nnz() >= (int64_t)INT32_MAX - 64) {
      err = "nnz must be below 2^31 on the device";
      return LP_ERR_INVALID;
    }
    const int m = h.m, n = h.n;
    const long long nnz = h.nnz();
    d->m = m;
    d->n = n;
    d->nnz = nnz;
    Layout L;
    const std::vector<TileShape> &cands = tile_candidates();
    build_layout(h, L, cands[kDefaultShape]);
    d->rperm = std::move(L.rperm);
    d->cperm = std::move(L.cperm);
    // the tile tables of every candidate shape (same row order, so one
    // stored matrix serves them all); the device buffers hold the largest
    {
      std::vector<int64_t> sa(m), st(n);
      for (int i = 0; i < m; ++i) sa[i] = L.arp[i + 1] - L.arp[i];
      for (int j = 0; j < n; ++j) st[j] = L.trp[j + 1] - L.trp[j];
      d->plansA.assign(cands.size(), TilePlan());
      d->plansT.assign(cands.size(), TilePlan());
      d->plansA[kDefaultShape] = std::move(L.pA);
      d->plansT[kDefaultShape] = std::move(L.pT);
      // the other candidates' plans, independent of one another, on host threads
      host_parallel_chunks(2 * cands.size(), nnz >= 1000000, [&](unsigned, size_t a, size_t b) {
        for (size_t q = a; q < b; ++q) {
          const size_t c = q / 2;
          if ((int)c == kDefaultShape) continue;
          if (q & 1) plan_tiles(st, cands[c], d->plansT[c]);
          else plan_tiles(sa, cands[c], d->plansA[c]);
        }
      });
    }
    size_t capTA = 1, capTT = 1, capSA = 1, capST = 1, capRA = 0, capRT = 0;
    int maxtiles = 0;
    for (size_t c = 0; c < cands.size(); ++c) {
      const TilePlan &a = d->plansA[c], &t = d->plansT[c];
      capTA = std::max(capTA, a.tiles.size());
      capTT = std::max(capTT, t.tiles.size());
      capSA = std::max(capSA, (size_t)a.seg_base.back());
      capST = std::max(capST, (size_t)t.seg_base.back());
      capRA = std::max(capRA, (size_t)a.nsegrows);
      capRT = std::max(capRT, (size_t)t.nsegrows);
      maxtiles = std::max(maxtiles, (int)std::max(a.tiles.size(), t.tiles.size()));
    }
    d->planA = d->planT = -1;
    d->bnorm = L.bnorm;
    d->cnorm = L.cnorm;
    d->off = L.off;
    // device buffers (value / index arrays padded past nnz)
    const size_t nzA = (size_t)nnz + kTilePad, nzT = (size_t)nnz + kTilePad;
    d->A_rp = d->dalloc_n<int>(m + 1);
    d->A_ci = d->dalloc_n<int>(nzA);
    d->A_v0 = d->dalloc_n<double>(nzA);
    d->A_v = d->dalloc_n<double>(nzA);
    d->T_rp = d->dalloc_n<int>(n + 1);
    d->T_ci = d->dalloc_n<int>(nzT);
    d->T_v0 = d->dalloc_n<double>(nzT);
    d->T_v = d->dalloc_n<double>(nzT);
    d->A_vf = d->dalloc_n<float>(nzA);
    d->T_vf = d->dalloc_n<float>(nzT);
    d->tilesA = d->dalloc_n<int2>(capTA);
    d->tilesT = d->dalloc_n<int2>(capTT);
    d->segbaseA = d->dalloc_n<int>(capRA + 1);
    d->segbaseT = d->dalloc_n<int>(capRT + 1);
    d->segcntA = d->dalloc_n<int>(std::max<size_t>(capRA, 1));
    d->segcntT = d->dalloc_n<int>(std::max<size_t>(capRT, 1));
    d->segpartA = d->dalloc_n<double>(capSA);
    d->segpartT = d->dalloc_n<double>(capST);
    double **cols_[] = {&d->c0, &d->lx0, &d->ux0, &d->c, &d->lx, &d->ux, &d->dc, &d->dc2,
                        &d->idc, &d->x, &d->x0, &d->xbar, &d->xhat, &d->zbuf, &d->pv,
                        &d->pv0, &d->pw, &d->ox, &d->oxi};
    for (double **p : cols_) *p = d->dalloc_n<double>(n);
    double **rows_[] = {&d->lc0, &d->uc0, &d->lc, &d->uc, &d->dr, &d->dr2, &d->idr, &d->y,
                        &d->y0, &d->yhat, &d->pu, &d->oy, &d->oyi};
    for (double **p : rows_) *p = d->dalloc_n<double>(m);
    d->dr_main = d->dr;
    d->dc_main = d->dc;
    d->xbar_f = d->dalloc_n<float2>(n);
    d->yf = d->dalloc_n<float2>(m);
    // the grid of each precision's solve: its iteration kernels' residency
    int occ64 = 1, occ32 = 1;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k_primal<double, true>, kBlock,
                                                     kSmem64));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_primal<float, true>, kBlock,
                                                     kSmem32));
    const int wpb = kBlock / 32;
    int need = (maxtiles + wpb - 1) / wpb;
    d->G64 = std::max(1, std::min(need, d->sm_count * std::max(occ64, 1)));
    d->G32 = std::max(1, std::min(need, d->sm_count * std::max(occ32, 1)));
    d->G = std::max(d->G64, d->G32);  // partials are sized for the larger
    // a quantity's partials: one per CTA, then one per segmented row (those
    // of the other matrix stay zero)
    d->GP = d->G + (int)std::max(capRA, capRT);
    d->partials = d->dalloc_n<double>((size_t)NQ * d->GP);
    d->st = d->dalloc_n<State>(1);
    CK(cudaMemcpyAsync(d->A_rp, L.arp.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->A_ci, L.aci.data(), sizeof(int) * nzA, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->A_v0, L.av.data(), sizeof(double) * nzA, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->T_rp, L.trp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->T_ci, L.tci.data(), sizeof(int) * nzT, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->T_v0, L.tv.data(), sizeof(double) * nzT, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemsetAsync(d->partials, 0, sizeof(double) * NQ * d->GP, d->s));
    CK(cudaMemsetAsync(d->segcntA, 0, sizeof(int) * std::max<size_t>(capRA, 1), d->s));
    CK(cudaMemsetAsync(d->segcntT, 0, sizeof(int) * std::max<size_t>(capRT, 1), d->s));
    install_plan(d, kDefaultShape, kDefaultShape);
    CK(cudaMemcpyAsync(d->c0, L.c0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->lx0, L.lx0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->ux0, L.ux0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->pv0, L.pv0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->lc0, L.lc0.data(), sizeof(double) * m, cudaMemcpyHostToDevice, d->s));
    CK(cudaMemcpyAsync(d->uc0, L.uc0.data(), sizeof(double) * m, cudaMemcpyHostToDevice, d->s));
    // the padding of the scaled copies is never used by the arithmetic, but
    // the tile copies read it: give it defined contents
    CK(cudaMemsetAsync(d->A_v, 0, sizeof(double) * nzA, d->s));
    CK(cudaMemsetAsync(d->T_v, 0, sizeof(double) * nzT, d->s));
    CK(cudaMemsetAsync(d->A_vf, 0, sizeof(float) * nzA, d->s));
    CK(cudaMemsetAsync(d->T_vf, 0, sizeof(float) * nzT, d->s));
    CK(cudaStreamSynchronize(d->s));
    d->uploaded = true;
  } catch (const DeviceOOM &e) {
    err = e.what();
    return LP_ERR_OOM;
  } catch (const std::exception &e) {
    err = e.what();
    return LP_ERR_CUDA;
  }
  return LP_OK;
}

namespace {

template <typename T>
void launch_primal(DeviceLP *d, bool wr, int grid, int j) {
  const T *va;
  size_t smem;
  if constexpr (sizeof(T) == 4) {
    va = reinterpret_cast<const T *>(d->T_vf);
    smem = kSmem32;
  } else {
    va = reinterpret_cast<const T *>(d->T_v);
    smem = kSmem64;
  }
  if (wr)
    k_primal<T, true><<<grid, kBlock, smem, d->s>>>(d->matT(), va, d->T_v, d->y, d->yf, d->c, d->lx,
                                                    d->ux, d->x, d->x0, d->xbar, d->xbar_f,
                                                    d->xhat, d->st, j, d->partials, d->GP);
  else
    k_primal<T, false><<<grid, kBlock, smem, d->s>>>(d->matT(), va, d->T_v, d->y, d->yf, d->c, d->lx,
                                                     d->ux, d->x, d->x0, d->xbar, d->xbar_f,
                                                     d->xhat, d->st, j, d->partials, d->GP);
}

template <typename T>
void launch_dual(DeviceLP *d, bool wr, int grid, int j) {
  const T *va;
  size_t smem;
  float2 *yf;
  if constexpr (sizeof(T) == 4) {
    va = reinterpret_cast<const T *>(d->A_vf);
    smem = kSmem32;
    yf = d->yf;
  } else {
    va = reinterpret_cast<const T *>(d->A_v);
    smem = kSmem64;
    yf = nullptr;
  }
  if (wr)
    k_dual<T, true><<<grid, kBlock, smem, d->s>>>(d->matA(), va, d->A_v, d->xbar, d->xbar_f, d->lc,
                                                  d->uc, d->y, d->y0, yf, d->yhat, d->st, j,
                                                  d->partials, d->GP);
  else
    k_dual<T, false><<<grid, kBlock, smem, d->s>>>(d->matA(), va, d->A_v, d->xbar, d->xbar_f, d->lc,
                                                   d->uc, d->y, d->y0, yf, d->yhat, d->st, j,
                                                   d->partials, d->GP);
}

void launch_kkt(DeviceLP *d, int force) {
  k_kkt_rows<<<d->G, kBlock, kSmem64, d->s>>>(d->matA(), d->A_v, d->xhat, d->dr, d->idr, d->lc0,
                                              d->uc0, d->yhat, d->st, force, d->partials, d->GP);
  k_kkt_cols<<<d->G, kBlock, kSmem64, d->s>>>(d->matT(), d->T_v, d->yhat, d->c, d->dc, d->idc,
                                              d->c0, d->lx0, d->ux0, d->xhat, d->zbuf, d->st,
                                              force, d->partials, d->GP);
}

// one PDHG iteration (position j in its chunk); check adds K3, K4, K5
void launch_iteration(DeviceLP *d, bool mixed, int j, bool check, bool hat_only) {
  const int gA = d->grid_tiles(d->ntilesA, d->nlongA);
  const int gT = d->grid_tiles(d->ntilesT, d->nlongT);
  const bool wr = check || hat_only;
  // kernels that write partials cover all G slots
  const int gT1 = wr ? d->G : gT;
  const int gA1 = wr ? d->G : gA;
  if (mixed) {
    launch_primal<float>(d, wr, gT1, j);
    launch_dual<float>(d, wr, gA1, j);
  } else {
    launch_primal<double>(d, wr, gT1, j);
    launch_dual<double>(d, wr, gA1, j);
  }
  d->launches += 2;
  if (check) {
    launch_kkt(d, 0);
    if (d->infeas_every > 0) {
      // pw (n) and pu (m) are the power iteration's vectors, free after set-up
      k_inf_prep<<<d->G, kBlock, 0, d->s>>>(d->st, d->n, d->xhat, d->x0, d->dc, d->c0, d->lx0,
                                            d->ux0, d->pw, d->partials, d->GP);
      k_inf_rows<<<d->G, kBlock, kSmem64, d->s>>>(d->matA(), d->A_v, d->pw, d->dr, d->idr,
                                                  d->lc0, d->uc0, d->yhat, d->y0, d->pu, d->st,
                                                  d->partials, d->GP);
      k_inf_cols<<<d->G, kBlock, kSmem64, d->s>>>(d->matT(), d->T_v, d->pu, d->idc, d->lx0,
                                                  d->ux0, d->st, d->partials, d->GP);
      d->launches += 3;
    }
    k_check<<<1, kBlock, 0, d->s>>>(d->st, d->partials, d->GP, 0);
    k_restart<<<d->grid_for(std::max(d->m, d->n)), kBlock, 0, d->s>>>(
        d->st, d->n, d->m, d->x, d->x0, d->xhat, d->y, d->y0, d->yhat, mixed ? d->yf : nullptr);
    d->launches += 4;
  }
}

void final_eval(DeviceLP *d) {
  launch_kkt(d, 1);
  k_check<<<1, kBlock, 0, d->s>>>(d->st, d->partials, d->GP, 1);
  d->launches += 3;
}

// ---- tile-shape autotuner of the grid engine -------------------------------
//
// Per matrix (rows of A for K2, rows of A^T for K1) the candidate shapes are
// timed on the first solve of a size class -- (log2 rows, 2 log2 mean row
// length, precision) -- with CUDA events around each kernel, 2 warm-up and
// 4 timed iterations per candidate, after the scaling and before the power
// iteration; the fastest is kept for the process.  The measured launches
// run the real iteration kernels on the scaled matrices from the start
// point; the set-up initialises the iterate and the state afterwards, so
// the solve itself is the same as with the chosen shape given in the options.

std::mutex g_tune_mu;
std::map<long long, int> g_tune_cache;

long long tune_key(int mat, long long rows, long long nnz, bool mixed) {
  const int rb = rows > 0 ? (int)std::floor(std::log2((double)rows)) : 0;
  const int lb =
      rows > 0 ? (int)std::floor(2.0 * std::log2(std::max(1.0, (double)nnz / (double)rows))) : 0;
  return ((long long)mat << 40) | ((long long)(mixed ? 1 : 0) << 32) | ((long long)rb << 16) |
         (long long)lb;
}

// measure: 0 = the cached choice or the default shape, 1 = measure on a miss
void tune_tiles(DeviceLP *d, bool mixed, bool measure) {
  const std::vector<TileShape> &cands = tile_candidates();
  const int nc = (int)cands.size();
  const long long kA = tune_key(0, d->m, d->nnz, mixed), kT = tune_key(1, d->n, d->nnz, mixed);
  d->tune_msA.clear();
  d->tune_msT.clear();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto a = g_tune_cache.find(kA), t = g_tune_cache.find(kT);
    if (a != g_tune_cache.end() && t != g_tune_cache.end()) {
      install_plan(d, a->second, t->second);
      return;
    }
  }
  if (!measure) {
    install_plan(d, kDefaultShape, kDefaultShape);
    return;
  }
  ScopedEvents owned;
  cudaEvent_t ev[3];
  for (cudaEvent_t &e : ev) e = owned.make();
  constexpr int kWarm = 2, kTimed = 4;
  d->tune_msA.assign(nc, 0.0);
  d->tune_msT.assign(nc, 0.0);
  for (int c = 0; c < nc; ++c) {
    install_plan(d, c, c);
    const int gA = d->grid_tiles(d->ntilesA, d->nlongA);
    const int gT = d->grid_tiles(d->ntilesT, d->nlongT);
    for (int r = 0; r < kWarm + kTimed; ++r) {
      CK(cudaEventRecord(ev[0], d->s));
      if (mixed) launch_primal<float>(d, false, gT, 1);
      else launch_primal<double>(d, false, gT, 1);
      CK(cudaEventRecord(ev[1], d->s));
      if (mixed) launch_dual<float>(d, false, gA, 1);
      else launch_dual<double>(d, false, gA, 1);
      CK(cudaEventRecord(ev[2], d->s));
      CK(cudaEventSynchronize(ev[2]));
      if (r >= kWarm) {
        float t1 = 0, t2 = 0;
        CK(cudaEventElapsedTime(&t1, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&t2, ev[1], ev[2]));
        d->tune_msT[c] += t1 / kTimed;
        d->tune_msA[c] += t2 / kTimed;
      }
    }
  }
  const int bA = (int)(std::min_element(d->tune_msA.begin(), d->tune_msA.end()) -
                       d->tune_msA.begin());
  const int bT = (int)(std::min_element(d->tune_msT.begin(), d->tune_msT.end()) -
                       d->tune_msT.begin());
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[kA] = bA;
    g_tune_cache[kT] = bT;
  }
  install_plan(d, bA, bT);
  d->launches += 2LL * (kWarm + kTimed) * nc;
}

// tune: 0 = keep the installed tile shapes, 1 = the cached choice or the
// default, 2 = also measure the candidates on a cache miss
void setup_device(DeviceLP *d, const lp_solve_opts &o, bool mixed, const double *xinit_perm,
                  const double *yinit_perm, int tune) {
  const int m = d->m, n = d->n;
  const int gm = d->grid_for(std::max(m, 1)), gn = d->grid_for(std::max(n, 1));
  const int gwm = d->grid_for((long long)std::max(m, 1) * 32);
  const int gwn = d->grid_for((long long)std::max(n, 1) * 32);
  k_fill<<<gm, kBlock, 0, d->s>>>(d->dr, 1.0, m);
  k_fill<<<gn, kBlock, 0, d->s>>>(d->dc, 1.0, n);
  d->launches += 2;
  for (int it = 0; it < o.ruiz_iters; ++it) {
    k_scale_pass<false, false><<<gwm, kBlock, 0, d->s>>>(m, d->A_rp, d->A_ci, d->A_v0, d->dr,
                                                         d->dc, d->dr2);
    k_scale_pass<true, false><<<gwn, kBlock, 0, d->s>>>(n, d->T_rp, d->T_ci, d->T_v0, d->dc,
                                                        d->dr, d->dc2);
    std::swap(d->dr, d->dr2);
    std::swap(d->dc, d->dc2);
    d->launches += 2;
  }
  if (o.pock_chambolle) {
    k_scale_pass<false, true><<<gwm, kBlock, 0, d->s>>>(m, d->A_rp, d->A_ci, d->A_v0, d->dr,
                                                        d->dc, d->dr2);
    k_scale_pass<true, true><<<gwn, kBlock, 0, d->s>>>(n, d->T_rp, d->T_ci, d->T_v0, d->dc,
                                                       d->dr, d->dc2);
    std::swap(d->dr, d->dr2);
    std::swap(d->dc, d->dc2);
    d->launches += 2;
  }
  // the ping-pong above may leave the result in the scratch buffers; the
  // captured iteration graph reads dr / dc from fixed addresses, so move the
  // final scales back to the canonical buffers
  if (d->dr != d->dr_main) {
    CK(cudaMemcpyAsync(d->dr_main, d->dr, sizeof(double) * std::max(m, 1),
                       cudaMemcpyDeviceToDevice, d->s));
    std::swap(d->dr, d->dr2);
  }
  if (d->dc != d->dc_main) {
    CK(cudaMemcpyAsync(d->dc_main, d->dc, sizeof(double) * std::max(n, 1),
                       cudaMemcpyDeviceToDevice, d->s));
    std::swap(d->dc, d->dc2);
  }
  k_apply_matrix<false><<<gwm, kBlock, 0, d->s>>>(m, d->A_rp, d->A_ci, d->A_v0, d->dr, d->dc,
                                                  d->A_v, mixed ? d->A_vf : nullptr);
  k_apply_matrix<true><<<gwn, kBlock, 0, d->s>>>(n, d->T_rp, d->T_ci, d->T_v0, d->dc, d->dr,
                                                 d->T_v, mixed ? d->T_vf : nullptr);
  k_apply_cols<<<d->G, kBlock, 0, d->s>>>(n, d->c0, d->lx0, d->ux0, d->dc, d->c, d->lx, d->ux,
                                          d->partials, d->GP);
  k_apply_rows<<<d->G, kBlock, 0, d->s>>>(m, d->lc0, d->uc0, d->dr, d->lc, d->uc, d->partials,
                                          d->GP);
  k_reciprocal<<<gm, kBlock, 0, d->s>>>(m, d->dr, d->idr);
  k_reciprocal<<<gn, kBlock, 0, d->s>>>(n, d->dc, d->idc);
  d->launches += 6;
  if (tune > 0) {
    // the measurement's iterations start from the initial point (set again
    // below); the state is still the host's initial copy (running, zero steps)
    k_init_x<<<gn, kBlock, 0, d->s>>>(n, d->lx, d->ux, d->dc, xinit_perm, d->x, d->x0);
    k_init_y<<<gm, kBlock, 0, d->s>>>(m, d->dr, yinit_perm, d->y, d->y0, mixed ? d->yf : nullptr);
    d->launches += 2;
    tune_tiles(d, mixed, tune == 2);
  }
  bool power = !(o.step_size > 0) && n > 0 && m > 0;
  if (power) {
    k_fill<<<gn, kBlock, 0, d->s>>>(d->pv, 1.0 / std::sqrt((double)n), n);
    d->launches += 1;
    const int gA = d->grid_tiles(d->ntilesA, d->nlongA);
    for (int it = 0; it < o.power_iters; ++it) {
      k_spmv_store<<<gA, kBlock, kSmem64, d->s>>>(d->matA(), d->A_v, d->pv, d->pu);
      k_spmv_store_sq<Q_PW><<<d->G, kBlock, kSmem64, d->s>>>(d->matT(), d->T_v, d->pu, d->pw,
                                                       d->partials, d->GP);
      k_normalize<<<gn, kBlock, 0, d->s>>>(n, d->pw, d->pv, d->pv0, d->partials, d->GP);
      d->launches += 3;
    }
    k_spmv_store_sq<Q_PWA><<<d->G, kBlock, kSmem64, d->s>>>(d->matA(), d->A_v, d->pv, d->pu,
                                                     d->partials, d->GP);
    d->launches += 1;
  }
  k_init_x<<<gn, kBlock, 0, d->s>>>(n, d->lx, d->ux, d->dc, xinit_perm, d->x, d->x0);
  k_init_y<<<gm, kBlock, 0, d->s>>>(m, d->dr, yinit_perm, d->y, d->y0, mixed ? d->yf : nullptr);
  k_setup_final<<<1, kBlock, 0, d->s>>>(d->st, d->partials, d->GP, o.step_size, o.primal_weight,
                                        power ? 1 : 0);
  d->launches += 3;
}

}  // namespace

void dev_tile_cache_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}

// the last solve's tile shapes and measurement (see lp_get_tile_tuning)
int dev_tile_tuning(const DeviceLP *d, double *out, int cap) {
  const std::vector<TileShape> &cands = tile_candidates();
  const int nc = (int)cands.size();
  if (cap < 3 + 4 * nc) return -1;
  out[0] = d->planA;
  out[1] = d->planT;
  out[2] = d->tune_msA.empty() ? 0.0 : 1.0;
  for (int c = 0; c < nc; ++c) {
    out[3 + 4 * c] = cands[c].run_max;
    out[4 + 4 * c] = cands[c].tile_nnz;
    out[5 + 4 * c] = d->tune_msA.empty() ? 0.0 : d->tune_msA[c];
    out[6 + 4 * c] = d->tune_msT.empty() ? 0.0 : d->tune_msT[c];
  }
  return 3 + 4 * nc;
}

int dev_solve(DeviceLP *d, const HostLP &h, const lp_solve_opts &o, lp_result *res,
              DeviceSolution &sol, std::string &err) {
  auto t_start = std::chrono::steady_clock::now();
  try {
    CK(cudaSetDevice(d->device));
    const bool mixed = o.precision == LP_MIXED;
    const int m = d->m, n = d->n;
    const int K = std::max(1, o.check_every);
    d->launches = 0;
    d->last_precision = o.precision;
    // this solve's grid (its precision's iteration-kernel residency); every
    // per-CTA and per-row partial slot starts clean
    d->G = mixed ? d->G32 : d->G64;
    CK(cudaMemsetAsync(d->partials, 0, sizeof(double) * NQ * (size_t)d->GP, d->s));
    // state constants
    State init{};
    init.rho = o.rho;
    init.beta_suff = o.beta_suff;
    init.beta_nec = o.beta_nec;
    init.beta_art = o.beta_art;
    init.theta = o.theta;
    init.eps_rel = o.eps_rel;
    init.eps_gap = o.eps_gap_rel > 0 ? o.eps_gap_rel : o.eps_rel;
    init.stop_on = 0;
    init.polish = o.polish ? 1 : 0;
    init.next_polish = 0;
    init.eps_infeas = o.eps_infeas;
    init.infeas_every = o.infeas_every;
    init.omega_clamp = o.primal_weight_clamp;
    d->infeas_every = o.infeas_every;
    init.bnorm = d->bnorm;
    init.cnorm = d->cnorm;
    init.off = d->off;
    init.K = K;
    init.halpern = o.halpern ? 1 : 0;
    init.restarts_on = o.restarts ? 1 : 0;
    init.status = ST_RUNNING;
    init.mixed_active = mixed ? 1 : 0;
    init.stall = 0;
    init.best_rel = INFINITY;
    init.t_switch = -1;
    CK(cudaMemcpyAsync(d->st, &init, sizeof(State), cudaMemcpyHostToDevice, d->s));
    // warm start, permuted to the device order
    double *xin = nullptr, *yin = nullptr;
    if (o.x_init || o.y_init) {
      if (d->hbuf) cudaFreeHost(d->hbuf);
      CK(cudaHostAlloc(reinterpret_cast<void **>(&d->hbuf), sizeof(double) * (size_t)(n + m + 2),
                       cudaHostAllocDefault));
      if (o.x_init) {
        for (int j = 0; j < n; ++j) d->hbuf[j] = o.x_init[d->cperm[j]];
        xin = d->ox;
        CK(cudaMemcpyAsync(xin, d->hbuf, sizeof(double) * n, cudaMemcpyHostToDevice, d->s));
      }
      if (o.y_init) {
        for (int i = 0; i < m; ++i) d->hbuf[n + i] = o.y_init[d->rperm[i]];
        yin = d->oy;
        CK(cudaMemcpyAsync(yin, d->hbuf + n, sizeof(double) * m, cudaMemcpyHostToDevice, d->s));
      }
    }
    ScopedEvents owned;
    const cudaEvent_t e0 = owned.make(), e1 = owned.make(), e2 = owned.make();
    CK(cudaEventRecord(e0, d->s));
    // tile shapes: given, or the autotuner's (measured after the set-up)
    const bool fixed_shape = o.tile_run_max > 0 && o.tile_nnz > 0;
    if (fixed_shape) {
      const int ci = tile_candidate_index(o.tile_run_max, o.tile_nnz);
      if (ci < 0) {
        err = "tile_run_max / tile_nnz is not a candidate shape";
        return LP_ERR_INVALID;
      }
      install_plan(d, ci, ci);
      d->tune_msA.clear();
      d->tune_msT.clear();
    }
    // k_setup_final overwrites the state's running fields; constants stay
    setup_device(d, o, mixed, xin, yin, fixed_shape ? 0 : (o.max_iter > 64 ? 2 : 1));
    CK(cudaGetLastError());
    CK(cudaEventRecord(e1, d->s));
    // iteration driver
    const long long max_iter = o.max_iter;
    int pi = mixed ? 1 : 0;
    bool use_graph = o.use_graph != 0;
    const int with_inf = d->infeas_every > 0 ? 1 : 0;
    if (use_graph &&
        (d->graph[pi] == nullptr || d->graph_K[pi] != K || d->graph_inf[pi] != with_inf)) {
      if (d->graph[pi]) {
        cudaGraphExecDestroy(d->graph[pi]);
        d->graph[pi] = nullptr;
      }
      cudaGraph_t g;
      long long saved = d->launches;
      CK(cudaStreamBeginCapture(d->s, cudaStreamCaptureModeThreadLocal));
      for (int j = 0; j < K; ++j) launch_iteration(d, mixed, j, j == 0, false);
      cudaMemcpyAsync(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost, d->s);
      CK(cudaStreamEndCapture(d->s, &g));
      CK(cudaGraphInstantiate(&d->graph[pi], g, 0));
      CK(cudaGraphDestroy(g));
      d->graph_K[pi] = K;
      d->graph_inf[pi] = with_inf;
      d->launches = saved;
    }
    const long long per_graph = 2LL * K + 4 + 3LL * with_inf;
    std::vector<cudaEvent_t> pool;
    auto get_event = [&]() {
      cudaEvent_t e;
      if (!pool.empty()) {
        e = pool.back();
        pool.pop_back();
      } else {
        e = owned.make(cudaEventDisableTiming);
      }
      return e;
    };
    bool timed_out = false;
    const double tl = o.time_limit_s > 0 ? o.time_limit_s : 1e30;
    // Run the state on the device from iteration `launched` until it leaves
    // ST_RUNNING (stops, or a check asks for polishing), `limit` iterations
    // have been launched, a bounded wait fails or the time limit passes;
    // then drain the stream.
    auto drive = [&](long long limit, long long &launched) {
      std::vector<cudaEvent_t> evs;
      size_t head = 0;
      for (;;) {
        // keep up to two chunks in flight
        while (evs.size() - head < 2 && launched < limit) {
          long long rem = limit - launched;
          if (use_graph && rem > K) {
            CK(cudaGraphLaunch(d->graph[pi], d->s));
            d->launches += per_graph;
            launched += K;
          } else {
            long long len = std::min<long long>(rem, K);
            for (long long j = 0; j < len; ++j) {
              bool last = (launched + j + 1 == limit);
              launch_iteration(d, mixed, (int)j, j == 0, last && j != 0);
            }
            CK(cudaMemcpyAsync(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost, d->s));
            launched += len;
          }
          cudaEvent_t e = get_event();
          CK(cudaEventRecord(e, d->s));
          evs.push_back(e);
        }
        if (head == evs.size()) break;
        CK(cudaEventSynchronize(evs[head]));
        pool.push_back(evs[head]);
        ++head;
        volatile int status = d->hst->status;
        {
          const State &V = *d->hst;
          trace_state("grid", V.t, V.rel_kkt, V.rel_p, V.rel_d, V.rel_gap, V.omega, V.restarts,
                      V.mixed_active);
        }
        if (o.verbose) {
          const State &V = *d->hst;
          std::fprintf(stderr, "pdhg t=%lld rel_kkt=%.3e rel_p=%.2e rel_d=%.2e gap=%.2e "
                       "omega=%.3e restarts=%d fp32=%d stop_on=%d\n", V.t, V.rel_kkt, V.rel_p,
                       V.rel_d, V.rel_gap, V.omega, V.restarts, V.mixed_active, V.stop_on);
        }
        if (status != ST_RUNNING) break;
        double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (el > tl) {
          timed_out = true;
          break;
        }
      }
      CK(cudaStreamSynchronize(d->s));
      for (size_t q = head; q < evs.size(); ++q) pool.push_back(evs[q]);
      CK(cudaMemcpy(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost));
    };
    long long launched = 0;
    long long polish_iters = 0;
    int polish_attempts = 0;
    bool polished = false;
    for (;;) {
      drive(max_iter, launched);
      if (d->hst->status != ST_POLISH || timed_out) break;
      // ---- feasibility polishing at the check t = S.t ----------------------
      const State S = *d->hst;
      const long long tc = S.t;
      ++polish_attempts;
      if (!d->bx) {
        d->bx = d->dalloc_n<double>(n);
        d->bx0 = d->dalloc_n<double>(n);
        d->bxh = d->dalloc_n<double>(n);
        d->bxp = d->dalloc_n<double>(n);
        d->by = d->dalloc_n<double>(m);
        d->by0 = d->dalloc_n<double>(m);
        d->byh = d->dalloc_n<double>(m);
      }
      auto copy = [&](double *dst, const double *src, int cnt) {
        if (cnt) CK(cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, d->s));
      };
      copy(d->bx, d->x, n);
      copy(d->bx0, d->x0, n);
      copy(d->bxh, d->xhat, n);
      copy(d->by, d->y, m);
      copy(d->by0, d->y0, m);
      copy(d->byh, d->yhat, m);
      const long long budget =
          (long long)K * std::max(1LL, (long long)std::ceil(o.polish_fraction * (double)tc / K));
      const int gmn = d->grid_for(std::max(std::max(m, n), 1));
      auto phase_state = [&](int stop_on) {
        State P = S;
        P.status = ST_RUNNING;
        P.stop_on = stop_on;
        P.polish = 0;
        P.next_polish = 0;
        P.infeas_every = 0;
        P.omega0 = S.omega;
        P.tau = S.eta / S.omega;
        P.sigma = S.eta * S.omega;
        P.r0 = P.r_prev = P.last_r = 0.0;
        P.t = 0;
        P.iters = 0;
        P.k_base = 0;
        P.k_off = 0;
        P.restarts = 0;
        P.restart_flag = 0;
        P.stall = 0;
        P.best_rel = INFINITY;
        P.t_switch = -1;
        CK(cudaMemcpyAsync(d->st, &P, sizeof(State), cudaMemcpyHostToDevice, d->s));
      };
      // iterations a phase took: to its stopping check, or its whole budget
      auto phase_iters = [&](long long lim) {
        return d->hst->status == ST_RUNNING ? lim : d->hst->iters;
      };
      auto restore_data = [&]() {
        k_apply_cols<<<d->G, kBlock, 0, d->s>>>(n, d->c0, d->lx0, d->ux0, d->dc, d->c, d->lx,
                                                d->ux, d->partials, d->GP);
        k_apply_rows<<<d->G, kBlock, 0, d->s>>>(m, d->lc0, d->uc0, d->dr, d->lc, d->uc,
                                                d->partials, d->GP);
        d->launches += 2;
      };
      // primal phase: c = 0, from (x^, 0), until rel_p <= eps_rel
      if (n) CK(cudaMemsetAsync(d->c, 0, sizeof(double) * n, d->s));
      k_set_point<<<gmn, kBlock, 0, d->s>>>(n, m, d->bxh, nullptr, d->x, d->x0, d->y, d->y0,
                                            mixed ? d->yf : nullptr);
      phase_state(1);
      d->launches += 1;
      long long lp_ = 0;
      drive(budget, lp_);
      const bool ok_p = d->hst->status == LP_OPTIMAL;
      polish_iters += phase_iters(budget);
      if (ok_p) copy(d->bxp, d->xhat, n);
      restore_data();
      bool ok_d = false;
      if (ok_p && !timed_out) {
        // dual phase: finite bounds 0, from (0, y^), until rel_d <= eps_rel
        k_zero_finite<<<d->G, kBlock, 0, d->s>>>(n, d->lx);
        k_zero_finite<<<d->G, kBlock, 0, d->s>>>(n, d->ux);
        k_zero_finite<<<d->G, kBlock, 0, d->s>>>(m, d->lc);
        k_zero_finite<<<d->G, kBlock, 0, d->s>>>(m, d->uc);
        k_set_point<<<gmn, kBlock, 0, d->s>>>(n, m, nullptr, d->byh, d->x, d->x0, d->y, d->y0,
                                              mixed ? d->yf : nullptr);
        d->launches += 5;
        phase_state(2);
        long long ld = 0;
        drive(budget, ld);
        ok_d = d->hst->status == LP_OPTIMAL;
        polish_iters += phase_iters(budget);
        restore_data();
      }
      if (ok_p && ok_d) {
        // the pair (x of the primal phase, y of the dual phase) on the
        // original LP; yhat holds the dual phase's y
        copy(d->xhat, d->bxp, n);
        State E = S;
        E.status = ST_RUNNING;
        CK(cudaMemcpyAsync(d->st, &E, sizeof(State), cudaMemcpyHostToDevice, d->s));
        final_eval(d);
        CK(cudaMemcpyAsync(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost, d->s));
        CK(cudaStreamSynchronize(d->s));
        const State &V = *d->hst;
        if (V.rel_p <= S.eps_rel && V.rel_d <= S.eps_rel && V.rel_gap <= S.eps_gap) {
          State F = V;
          F.status = LP_OPTIMAL;
          F.iters = tc + 1;
          CK(cudaMemcpyAsync(d->st, &F, sizeof(State), cudaMemcpyHostToDevice, d->s));
          copy(d->x, d->bx, n);  // the returned iterate z^t stays the main one
          copy(d->y, d->by, m);
          CK(cudaStreamSynchronize(d->s));
          *d->hst = F;
          polished = true;
          break;
        }
      }
      // failed: the main state back, then the rest of the check at tc and of
      // its period
      copy(d->x, d->bx, n);
      copy(d->x0, d->bx0, n);
      copy(d->xhat, d->bxh, n);
      copy(d->y, d->by, m);
      copy(d->y0, d->by0, m);
      copy(d->yhat, d->byh, m);
      if (mixed && m) {
        k_split_y<<<gmn, kBlock, 0, d->s>>>(m, d->y, d->yf);
        d->launches += 1;
      }
      CK(cudaMemcpyAsync(d->st, &S, sizeof(State), cudaMemcpyHostToDevice, d->s));
      k_check_resume<<<1, 32, 0, d->s>>>(d->st);
      k_restart<<<d->grid_for(std::max(m, n)), kBlock, 0, d->s>>>(
          d->st, n, m, d->x, d->x0, d->xhat, d->y, d->y0, d->yhat, mixed ? d->yf : nullptr);
      d->launches += 2;
      const long long rest = std::min<long long>(K - 1, max_iter - 1 - tc);
      for (long long j = 1; j <= rest; ++j)
        launch_iteration(d, mixed, (int)j, false, tc + j + 1 == max_iter);
      launched = tc + 1 + std::max(0LL, rest);
      CK(cudaMemcpyAsync(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost, d->s));
      CK(cudaStreamSynchronize(d->s));
      if (d->hst->status != ST_RUNNING) break;
    }
    CK(cudaMemcpy(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost));
    int status = d->hst->status;
    long long iters = d->hst->iters;
    if (status == ST_RUNNING || status == ST_POLISH) {
      if (timed_out) {
        status = LP_TIME_LIMIT;
        iters = std::min(launched, max_iter);
        State fix = *d->hst;
        fix.status = LP_TIME_LIMIT;
        CK(cudaMemcpyAsync(d->st, &fix, sizeof(State), cudaMemcpyHostToDevice, d->s));
      } else {
        // max_iter reached: evaluate the last T(z)
        final_eval(d);
        status = LP_ITER_LIMIT;
        iters = max_iter;
      }
    } else if (status == LP_ITER_LIMIT) {
      iters = max_iter;
    }
    CK(cudaEventRecord(e2, d->s));
    // outputs
    const int gmn = d->grid_for(std::max(std::max(m, n), 1));
    k_unscale<<<gmn, kBlock, 0, d->s>>>(n, m, d->dc, d->dr, d->xhat, d->yhat, d->x, d->y, d->ox,
                                        d->oy, d->oxi, d->oyi);
    d->launches += 1;
    CK(cudaGetLastError());
    std::vector<double> hx(n), hy(m), hz(n), hxi(n), hyi(m);
    if (n) {
      CK(cudaMemcpyAsync(hx.data(), d->ox, sizeof(double) * n, cudaMemcpyDeviceToHost, d->s));
      CK(cudaMemcpyAsync(hxi.data(), d->oxi, sizeof(double) * n, cudaMemcpyDeviceToHost, d->s));
      CK(cudaMemcpyAsync(hz.data(), d->zbuf, sizeof(double) * n, cudaMemcpyDeviceToHost, d->s));
    }
    if (m) {
      CK(cudaMemcpyAsync(hy.data(), d->oy, sizeof(double) * m, cudaMemcpyDeviceToHost, d->s));
      CK(cudaMemcpyAsync(hyi.data(), d->oyi, sizeof(double) * m, cudaMemcpyDeviceToHost, d->s));
    }
    CK(cudaMemcpyAsync(d->hst, d->st, sizeof(State), cudaMemcpyDeviceToHost, d->s));
    CK(cudaStreamSynchronize(d->s));
    float ms_setup = 0, ms_solve = 0;
    CK(cudaEventElapsedTime(&ms_setup, e0, e1));
    CK(cudaEventElapsedTime(&ms_solve, e1, e2));
    sol.x.assign(n, 0.0);
    sol.z.assign(n, 0.0);
    sol.xi.assign(n, 0.0);
    sol.y.assign(m, 0.0);
    sol.yi.assign(m, 0.0);
    const bool par = d->nnz >= 1000000;
    host_parallel_chunks((size_t)n, par, [&](unsigned, size_t j0, size_t j1) {
      for (size_t j = j0; j < j1; ++j) {
        const int o2 = d->cperm[j];
        sol.x[o2] = hx[j];
        sol.xi[o2] = hxi[j];
        sol.z[o2] = hz[j];
      }
    });
    host_parallel_chunks((size_t)m, par, [&](unsigned, size_t i0, size_t i1) {
      for (size_t i = i0; i < i1; ++i) {
        const int o2 = d->rperm[i];
        sol.y[o2] = hy[i];
        sol.yi[o2] = hyi[i];
      }
    });
    sol.valid = true;
    const State &S = *d->hst;
    if (res) {
      res->termination = status;
      res->restarts = S.restarts;
      res->iterations = iters;
      res->rel_kkt = S.rel_kkt;
      res->rel_p = S.rel_p;
      res->rel_d = S.rel_d;
      res->rel_gap = S.rel_gap;
      res->r_p = S.r_p;
      res->r_d = S.r_d;
      res->gap = S.gap;
      res->primal_obj = S.pobj;
      res->dual_obj = S.dobj;
      res->eta = S.eta;
      res->omega = S.omega;
      res->t_setup_s = ms_setup * 1e-3;
      res->t_solve_s = ms_solve * 1e-3;
      res->t_total_s =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      res->kernel_launches = d->launches;
      res->fp32_iterations = mixed ? (S.t_switch >= 0 ? S.t_switch : iters) : 0;
      res->iterations = iters + polish_iters;
      res->polish_attempts = polish_attempts;
      res->polished = polished ? 1 : 0;
      res->polish_iterations = polish_iters;
    }
  } catch (const DeviceOOM &e) {
    err = e.what();
    return LP_ERR_OOM;
  } catch (const std::exception &e) {
    err = e.what();
    return LP_ERR_CUDA;
  }
  return LP_OK;
}

// Time the iteration kernels one launch at a time with CUDA events on the
// library's stream, each launch preceded by a write of a 256 MiB buffer so it
// starts with a cold L2.  Needs a prior dev_solve (scaled matrices present);
// perturbs the internal iterate (not the returned solution).
// out: [K1 ms, K2 ms, K1 bytes, K2 bytes, K3a ms, K3b ms, K3a bytes, K3b bytes]
int dev_profile(DeviceLP *d, int reps, double *out, std::string &err) {
  try {
    CK(cudaSetDevice(d->device));
    if (d->last_precision < 0) {
      err = "profile needs a prior solve";
      return LP_ERR_STATE;
    }
    const bool mixed = d->last_precision == LP_MIXED;
    const int m = d->m, n = d->n;
    const double nnz = (double)d->nnz;
    if (!d->flush) {
      d->flush_bytes = size_t(256) << 20;
      d->flush = d->dalloc(d->flush_bytes);
    }
    State saved;
    CK(cudaMemcpyAsync(&saved, d->st, sizeof(State), cudaMemcpyDeviceToHost, d->s));
    CK(cudaStreamSynchronize(d->s));
    State run = saved;
    run.status = ST_RUNNING;
    run.mixed_active = mixed ? 1 : 0;  // time the FP32 SpMV of a mixed solve
    CK(cudaMemcpyAsync(d->st, &run, sizeof(State), cudaMemcpyHostToDevice, d->s));
    CK(cudaStreamSynchronize(d->s));
    ScopedEvents owned;
    const cudaEvent_t a = owned.make(), b = owned.make();
    double tot[4] = {0, 0, 0, 0};
    const int gA = d->grid_tiles(d->ntilesA, d->nlongA);
    const int gT = d->grid_tiles(d->ntilesT, d->nlongT);
    for (int r = 0; r < reps; ++r) {
      for (int which = 0; which < 4; ++which) {
        CK(cudaMemsetAsync(d->flush, r & 0xff, d->flush_bytes, d->s));
        CK(cudaEventRecord(a, d->s));
        if (which == 0) {
          if (mixed) launch_primal<float>(d, false, gT, 1);
          else launch_primal<double>(d, false, gT, 1);
        } else if (which == 1) {
          if (mixed) launch_dual<float>(d, false, gA, 1);
          else launch_dual<double>(d, false, gA, 1);
        } else if (which == 2) {
          k_kkt_rows<<<d->G, kBlock, kSmem64, d->s>>>(d->matA(), d->A_v, d->xhat, d->dr, d->idr,
                                                      d->lc0, d->uc0, d->yhat, d->st, 1,
                                                      d->partials, d->GP);
        } else {
          k_kkt_cols<<<d->G, kBlock, kSmem64, d->s>>>(d->matT(), d->T_v, d->yhat, d->c, d->dc,
                                                      d->idc, d->c0, d->lx0, d->ux0, d->xhat,
                                                      d->zbuf, d->st, 1, d->partials, d->GP);
        }
        CK(cudaEventRecord(b, d->s));
        CK(cudaEventSynchronize(b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a, b));
        tot[which] += ms;
      }
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(d->st, &saved, sizeof(State), cudaMemcpyHostToDevice, d->s));
    CK(cudaStreamSynchronize(d->s));
    // algorithmic bytes: matrix values + column indices + row offsets, each
    // gathered vector counted once, every epilogue vector read / written once
    const double sv = mixed ? 4.0 : 8.0;
    const double sg = mixed ? 4.0 : 8.0;  // gathered vector element
    // K1 reads x, x0, c, lx, ux and writes x and xbar (4 bytes when mixed)
    const double k1 = nnz * (sv + 4.0) + 4.0 * (n + 1) + sg * m + 8.0 * 5 * n + 8.0 * n +
                      (mixed ? 4.0 : 8.0) * n;
    // K2 reads y, y0, lc, uc and writes y (+ its FP32 shadow when mixed)
    const double k2 = nnz * (sv + 4.0) + 4.0 * (m + 1) + sg * n + 8.0 * 4 * m + 8.0 * m +
                      (mixed ? 4.0 * m : 0.0);
    const double k3a = nnz * 12.0 + 4.0 * (m + 1) + 8.0 * n + 8.0 * 6 * m;
    const double k3b = nnz * 12.0 + 4.0 * (n + 1) + 8.0 * m + 8.0 * 8 * n + 8.0 * n;
    out[0] = tot[0] / reps;
    out[1] = tot[1] / reps;
    out[2] = k1;
    out[3] = k2;
    out[4] = tot[2] / reps;
    out[5] = tot[3] / reps;
    out[6] = k3a;
    out[7] = k3b;
  } catch (const std::exception &e) {
    err = e.what();
    return LP_ERR_CUDA;
  }
  return LP_OK;
}

}  // namespace gb300lp
