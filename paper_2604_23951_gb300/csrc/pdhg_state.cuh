// Per-LP PDHG state and the restart / termination decision shared by the
// single-LP path (solver.cu) and the batched path (batch.cu).
//
// The decision follows the solver reading documented with the oracle:
// checks at t = 0, K, 2K, ...; stop when T(z) passes the stopping test
// (rel_p, rel_d <= eps_rel and rel_gap <= eps_gap: with eps_gap = eps_rel,
// relative KKT error <= eps_rel) or a value is not finite; with
// r = ||z - T(z)||_omega,
// record r0 = r_prev = r at the first check, otherwise restart when
// r <= beta_suff r0, or r <= beta_nec r0 and r > r_prev, or k >= beta_art t;
// a restart moves the anchor and the iterate to T(z) and smooths the primal
// weight omega <- exp(theta log(dy / dx) + (1 - theta) log omega), kept
// within [omega_0 / clamp, omega_0 * clamp] when omega_clamp > 0.  At every
// infeas_every-th check that does not stop, the direction T(z) - z0 is
// tested for a dual ray (LP_INFEASIBLE) and then a primal ray
// (LP_UNBOUNDED), from the Q_I* quantities.
#pragma once

#include <cuda_runtime.h>

namespace gb300lp {

constexpr int ST_RUNNING = -1;
constexpr int ST_POLISH = -2;  // a check asked the host for feasibility polishing

// reduced quantities of a check (and of the set-up)
// Q_I*: infeasibility test of the direction (d, w) = T(z) - z0 (unscaled):
// c^T d, squared cone violations of d (columns) and A d (rows), squared
// residual ||A^T w + lam||^2, dual-ray objective (rows, columns)
enum {
  Q_XRES = 0, Q_XD, Q_YRES, Q_YD, Q_RP, Q_RDY, Q_DY, Q_RD, Q_DL, Q_P,
  Q_ICD, Q_IPVC, Q_IPVR, Q_IDR, Q_IDOR, Q_IDOC,
  Q_CN, Q_BN, Q_PW, Q_PWA, NQ
};
// (Q_PW: ||A^T A v||^2 of the power iteration's A^T passes; Q_PWA: ||A v||^2
// of its final pass over A.  Every quantity is summed from one matrix's
// kernels only, so the per-row slots of segmented rows never mix matrices.)


struct State {
  double eta, omega, tau, sigma;
  double rho, beta_suff, beta_nec, beta_art, theta, eps_rel;
  double eps_infeas;
  int infeas_every;  // 0: no infeasibility test
  double omega0, omega_clamp;  // initial primal weight; band factor (0: none)
  double r0, r_prev, last_r;
  double bnorm, cnorm, off;
  double rel_kkt, rel_p, rel_d, rel_gap, r_p, r_d, gap, pobj, dobj;
  long long t;
  long long iters;
  int K;
  int k_base, k_off;
  int restarts;
  int status;
  int restart_flag;
  int halpern, restarts_on;
  // mixed precision: 1 while the SpMV runs on FP32 matrix values; the check
  // switches the LP to the FP64 SpMV for good once the best rel-KKT so far
  // has not halved for kMixedStall checks
  int mixed_active;
  int stall;       // checks since the best rel-KKT halved
  double best_rel;
  long long t_switch;  // iteration of the FP64 switch (or -1)
  // stopping test: stop_on 0: rel_p <= eps_rel, rel_d <= eps_rel and rel_gap
  // <= eps_gap; 1: rel_p <= eps_rel only; 2: rel_d <= eps_rel only (the
  // phases of feasibility polishing)
  double eps_gap;
  int stop_on;
  // feasibility polishing: a check at t >= next_polish that does not stop,
  // with rel_gap <= eps_gap and rel_p or rel_d > eps_rel, saves its
  // quantities in pq and ends in ST_POLISH; the host runs the phases and
  // either finishes or resumes the check (check_update again, next_polish
  // = 2t)
  int polish;
  long long next_polish;
  double pq[NQ];
  long long dev_ns;  // batched slots: device time the slot's cluster spent on it
};

// FP64 switch of the mixed mode, a guard only: the mixed SpMV (FP32 matrix
// values, gathered vectors as float pairs, compensated accumulation) follows
// the FP64 trajectory to below 1e-7 on the planted power-law and presolvable
// structures -- rounding the matrix values to float perturbs the iteration
// little, while rounding the gathered vectors to float (an earlier form of
// this mode) stalled it between 1e-5 and 1e-6 -- so it runs to the
// tolerance unless its progress stops.
constexpr int kMixedStall = 256;

// whether the check at iteration t tests for infeasibility
__host__ __device__ __forceinline__ bool infeas_due(long long t, int K, int every) {
  return every > 0 && ((t / K) % every) == 0;
}

// Halpern coefficients of iteration position j of a check period:
// z+ = a T(z) + b z + g z0
struct Halpern {
  double a, b, g;
};
__device__ __forceinline__ Halpern halpern_coeffs(const State *st, int j) {
  double lam = 1.0;
  if (st->halpern) {
    int k = (j == 0) ? st->k_base : st->k_off + j;
    lam = (k + 1.0) / (k + 2.0);
  }
  Halpern h;
  h.a = lam * (1.0 + st->rho);
  h.b = -lam * st->rho;
  h.g = 1.0 - lam;
  return h;
}

// One thread: fold the check quantities q[0..Q_P] into st.  eval_only: fill
// in the KKT fields and mark LP_ITER_LIMIT (1) if still running.
__device__ __forceinline__ void check_update(State *st, const double *q, bool eval_only) {
  double rp = sqrt(q[Q_RP]);
  double rd = sqrt(q[Q_RD] + q[Q_RDY]);
  double p = q[Q_P] + st->off;
  double d = q[Q_DY] + q[Q_DL] + st->off;
  double relp = rp / (1.0 + st->bnorm);
  double reld = rd / (1.0 + st->cnorm);
  double gap = fabs(p - d);
  double relg = gap / (1.0 + fabs(p) + fabs(d));
  double rel = fmax(relp, fmax(reld, relg));
  st->rel_kkt = rel;
  st->rel_p = relp;
  st->rel_d = reld;
  st->rel_gap = relg;
  st->r_p = rp;
  st->r_d = rd;
  st->gap = gap;
  st->pobj = p;
  st->dobj = d;
  if (eval_only) {
    if (st->status == ST_RUNNING) st->status = 1;  // LP_ITER_LIMIT
    return;
  }
  bool finite = isfinite(rel) && isfinite(q[Q_XRES]) && isfinite(q[Q_YRES]);
  const bool met = st->stop_on == 1   ? relp <= st->eps_rel
                   : st->stop_on == 2 ? reld <= st->eps_rel
                                      : (relp <= st->eps_rel && reld <= st->eps_rel &&
                                         relg <= st->eps_gap);
  if (!finite || met) {
    st->status = finite ? 0 : 3;  // LP_OPTIMAL : LP_NUMERICAL
    st->iters = st->t + 1;
    st->restart_flag = 0;
    return;
  }
  if (infeas_due(st->t, st->K, st->infeas_every)) {
    const double dobj = q[Q_IDOR] + q[Q_IDOC];
    const double cd = q[Q_ICD];
    int cert = -1;
    if (dobj > 0 && sqrt(q[Q_IDR]) <= st->eps_infeas * dobj) cert = 4;  // LP_INFEASIBLE
    else if (cd < 0 && sqrt(q[Q_IPVC] + q[Q_IPVR]) <= st->eps_infeas * (-cd))
      cert = 5;  // LP_UNBOUNDED
    if (cert >= 0) {
      st->status = cert;
      st->iters = st->t + 1;
      st->restart_flag = 0;
      return;
    }
  }
  if (st->polish && st->stop_on == 0 && st->t >= st->next_polish && relg <= st->eps_gap &&
      fmax(relp, reld) > st->eps_rel) {
    for (int i = 0; i < NQ; ++i) st->pq[i] = q[i];
    st->status = ST_POLISH;
    st->restart_flag = 0;
    return;
  }
  if (st->mixed_active) {
    if (rel < 0.5 * st->best_rel) {
      st->best_rel = rel;
      st->stall = 0;
    } else {
      st->stall += 1;
    }
    if (st->stall >= kMixedStall) {
      st->mixed_active = 0;
      st->t_switch = st->t;
    }
  }
  double om = st->omega;
  double r = sqrt(om * q[Q_XRES] + q[Q_YRES] / om);
  st->last_r = r;
  int kb = st->k_base;
  int restart = 0;
  if (kb == 0) {
    st->r0 = st->r_prev = r;
  } else if (st->restarts_on &&
             (r <= st->beta_suff * st->r0 || (r <= st->beta_nec * st->r0 && r > st->r_prev) ||
              (double)kb >= st->beta_art * (double)st->t)) {
    double dx = sqrt(q[Q_XD]), dy = sqrt(q[Q_YD]);
    if (dx > 1e-10 && dy > 1e-10) om = exp(st->theta * log(dy / dx) + (1.0 - st->theta) * log(om));
    if (st->omega_clamp > 0.0)
      om = fmin(fmax(om, st->omega0 / st->omega_clamp), st->omega0 * st->omega_clamp);
    st->omega = om;
    st->tau = st->eta / om;
    st->sigma = st->eta * om;
    st->r0 = st->r_prev = r;
    st->restarts += 1;
    restart = 1;
  } else {
    st->r_prev = r;
  }
  st->restart_flag = restart;
  st->k_off = restart ? -1 : kb;
  st->k_base = st->k_off + st->K;
  st->t += st->K;
}

}  // namespace gb300lp
