// Per-row epilogues of the PDHG SpMVs (used with warp_spmv of
// spmv_warp.cuh by the single-LP kernels and by the batched cluster kernel).
//
// Every epilogue gets pre(r) (prefetch of the row's own vector entries, so
// those loads overlap the row's gathers) and then row(r, s) with
// s = (row r of the matrix) . vec, on the same thread.  Vectors are in the
// renumbered (length-sorted) order of the device layout.  clear() zeroes the
// accumulators and sink(k, r) stores them into slot r of their quantities
// (segmented rows: the warp that finishes the row runs the epilogue on a
// copy, so its contribution lands in a slot of the row's own).
#pragma once

#include "device_common.cuh"
#include "pdhg_state.cuh"
#include "spmv_warp.cuh"

namespace gb300lp {

// out[r] = s (power iteration); acc collects sum s^2
template <typename O, int QI = Q_PW>
struct StoreSqEpi {
  O *out;
  double acc;
  __device__ __forceinline__ void pre(int) {}
  __device__ __forceinline__ void row(int r, double s) {
    out[r] = (O)s;
    acc += s * s;
  }
  __device__ __forceinline__ void clear() { acc = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (k.p) k.p[QI * k.stride + k.base + r] = acc;
  }
};

// K1: g = (A~^T y)_j; primal half of the operator T (eq. for the primal
// step of PDHG), the reflection xbar = 2 xh - x and the Halpern update of x.
// CHECK: also store xh and collect ||x - xh||^2 and ||xh - x0||^2.
template <bool CHECK, bool MIXED>
struct PrimalEpi {
  const double *c, *lx, *ux;
  double *x, *x0, *xbar, *xhat;
  float2 *xbar_f;  // mixed: xbar as a float pair (split_f2) for the FP32 SpMV
  double tau;
  Halpern hc;
  double acc0, acc1;
  double xk, cj, lo, hi, a0;
  __device__ __forceinline__ void pre(int j) {
    xk = x[j];
    cj = c[j];
    lo = lx[j];
    hi = ux[j];
    a0 = x0[j];
  }
  __device__ __forceinline__ void row(int j, double g) {
    const double xh = clampd(fma(-tau, cj - g, xk), lo, hi);
    const double xb = fma(2.0, xh, -xk);
    x[j] = fma(hc.a, xh, fma(hc.b, xk, hc.g * a0));
    if (MIXED) xbar_f[j] = split_f2(xb); else xbar[j] = xb;
    if (CHECK) {
      xhat[j] = xh;
      acc0 += (xk - xh) * (xk - xh);
      acc1 += (xh - a0) * (xh - a0);
    }
  }
  __device__ __forceinline__ void clear() { acc0 = acc1 = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (CHECK && k.p) {
      k.p[Q_XRES * k.stride + k.base + r] = acc0;
      k.p[Q_XD * k.stride + k.base + r] = acc1;
    }
  }
};

// K2: h = (A~ xbar)_i; dual half of T with the division-free prox
// v + sigma proj_[l,u](-v / sigma) = v + proj_[sigma l, sigma u](-v), and the
// Halpern update of y.
template <bool CHECK, bool MIXED>
struct DualEpi {
  const double *lc, *uc;
  double *y, *y0, *yhat;
  float2 *yf;  // mixed: y as a float pair
  double sigma;
  Halpern hc;
  double acc0, acc1;
  double yk, lo, hi, a0;
  __device__ __forceinline__ void pre(int i) {
    yk = y[i];
    lo = lc[i];
    hi = uc[i];
    a0 = y0[i];
  }
  __device__ __forceinline__ void row(int i, double h) {
    const double v = fma(-sigma, h, yk);
    const double yh = v + clampd(-v, sigma * lo, sigma * hi);
    const double yn = fma(hc.a, yh, fma(hc.b, yk, hc.g * a0));
    y[i] = yn;
    if (MIXED) yf[i] = split_f2(yn);
    if (CHECK) {
      yhat[i] = yh;
      acc0 += (yk - yh) * (yk - yh);
      acc1 += (yh - a0) * (yh - a0);
    }
  }
  __device__ __forceinline__ void clear() { acc0 = acc1 = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (CHECK && k.p) {
      k.p[Q_YRES * k.stride + k.base + r] = acc0;
      k.p[Q_YD * k.stride + k.base + r] = acc1;
    }
  }
};

// K3a: rows of A at xh: primal residual of the unscaled A x against
// [l_c, u_c], the y-domain violation and the y part of the dual objective
struct KktRowEpi {
  const double *dr, *idr, *lc0, *uc0, *yhat;
  double rp2, rdy2, dy;
  __device__ __forceinline__ void pre(int) {}
  __device__ __forceinline__ void row(int i, double h) {
    const double ax = h * idr[i];
    const double lo = lc0[i], hi = uc0[i];
    const double pr = clampd(ax, lo, hi);
    rp2 += (ax - pr) * (ax - pr);
    const double yv = dr[i] * yhat[i];
    double yp = yv;
    if (!isfinite(lo)) yp = fmin(yp, 0.0);
    if (!isfinite(hi)) yp = fmax(yp, 0.0);
    rdy2 += (yv - yp) * (yv - yp);
    dy += support_term(yp, lo, hi);
  }
  __device__ __forceinline__ void clear() { rp2 = rdy2 = dy = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (!k.p) return;
    k.p[Q_RP * k.stride + k.base + r] = rp2;
    k.p[Q_RDY * k.stride + k.base + r] = rdy2;
    k.p[Q_DY * k.stride + k.base + r] = dy;
  }
};

// K3b: rows of A^T at yh: reduced costs c - A^T y (unscaled, stored in zbuf),
// the dual residual, the lambda part of the dual objective and c^T x
struct KktColEpi {
  const double *c, *dc, *idc, *c0, *lx0, *ux0, *xhat;
  double *zbuf;
  double rd2, dl, p;
  __device__ __forceinline__ void pre(int) {}
  __device__ __forceinline__ void row(int j, double h) {
    const double d = dc[j];
    const double g = (c[j] - h) * idc[j];
    const double lo = lx0[j], hi = ux0[j];
    const bool lf = isfinite(lo), uf = isfinite(hi);
    double lam = g;
    if (!lf && !uf) lam = 0.0;
    else if (lf && !uf) lam = fmax(lam, 0.0);
    else if (!lf && uf) lam = fmin(lam, 0.0);
    rd2 += (g - lam) * (g - lam);
    dl += support_term(lam, lo, hi);
    p += c0[j] * (d * xhat[j]);
    zbuf[j] = g;
  }
  __device__ __forceinline__ void clear() { rd2 = dl = p = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (!k.p) return;
    k.p[Q_RD * k.stride + k.base + r] = rd2;
    k.p[Q_DL * k.stride + k.base + r] = dl;
    k.p[Q_P * k.stride + k.base + r] = p;
  }
};

// Infeasibility test, rows of A at d~ = xh - x0 (scaled): squared violation
// of A d (unscaled) against the recession cone of [l_c, u_c] ((A d)_i <= 0
// where u_ci is finite, >= 0 where l_ci is); the dual direction
// w~ = yh - y0 projected on the rows' sign domain (stored in wbuf for the
// A^T pass) and its part of the dual-ray objective sum(w+ l_c - w- u_c)
struct InfRowEpi {
  const double *dr, *idr, *lc0, *uc0, *yhat, *y0;
  double *wbuf;
  double v2, dobj;
  __device__ __forceinline__ void pre(int) {}
  __device__ __forceinline__ void row(int i, double h) {
    const double ad = h * idr[i];
    const double lo = lc0[i], hi = uc0[i];
    const bool lf = isfinite(lo), uf = isfinite(hi);
    double v = 0.0;
    if (uf) v += fmax(ad, 0.0);
    if (lf) v += fmax(-ad, 0.0);
    v2 += v * v;
    double w = yhat[i] - y0[i];
    if (!lf) w = fmin(w, 0.0);
    if (!uf) w = fmax(w, 0.0);
    wbuf[i] = w;
    dobj += support_term(dr[i] * w, lo, hi);
  }
  __device__ __forceinline__ void clear() { v2 = dobj = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (!k.p) return;
    k.p[Q_IPVR * k.stride + k.base + r] = v2;
    k.p[Q_IDOR * k.stride + k.base + r] = dobj;
  }
};

// Infeasibility test, rows of A^T at the projected w~: g = A^T w (unscaled),
// lam = proj_Lambda(-g), the squared residual (g + lam)^2 and the column part
// of the dual-ray objective sum(lam+ l_x - lam- u_x)
struct InfColEpi {
  const double *idc, *lx0, *ux0;
  double r2, dobj;
  __device__ __forceinline__ void pre(int) {}
  __device__ __forceinline__ void row(int j, double h) {
    const double g = h * idc[j];
    const double lo = lx0[j], hi = ux0[j];
    const bool lf = isfinite(lo), uf = isfinite(hi);
    double lam = -g;
    if (!lf && !uf) lam = 0.0;
    else if (lf && !uf) lam = fmax(lam, 0.0);
    else if (!lf && uf) lam = fmin(lam, 0.0);
    r2 += (g + lam) * (g + lam);
    dobj += support_term(lam, lo, hi);
  }
  __device__ __forceinline__ void clear() { r2 = dobj = 0.0; }
  __device__ __forceinline__ void sink(const AccSink &k, int r) const {
    if (!k.p) return;
    k.p[Q_IDR * k.stride + k.base + r] = r2;
    k.p[Q_IDOC * k.stride + k.base + r] = dobj;
  }
};

// Infeasibility test, one column: d~_j = xh_j - x0_j (stored in dbuf for the
// A pass); c^T d and the squared violation of d (unscaled) against the
// recession cone of [l_x, u_x]
__device__ __forceinline__ void inf_col_prep(int j, const double *xhat, const double *x0,
                                             const double *dc, const double *c0,
                                             const double *lx0, const double *ux0, double *dbuf,
                                             double &cd, double &v2) {
  const double dd = xhat[j] - x0[j];
  dbuf[j] = dd;
  const double d = dc[j] * dd;
  cd += c0[j] * d;
  double v = 0.0;
  if (isfinite(ux0[j])) v += fmax(d, 0.0);
  if (isfinite(lx0[j])) v += fmax(-d, 0.0);
  v2 += v * v;
}

}  // namespace gb300lp
