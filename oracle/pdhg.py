"""Oracle PDHG for  min c^T x  s.t.  l_c <= A x <= u_c,  l_x <= x <= u_x  (eq. (1)).

TEST INFRASTRUCTURE ONLY (see the package header).  FP64 throughout.

The paper (Sec. 1 and Sec. 4.2) names the solver it times -- a restarted PDHG
method in the PDLP / cuPDLP / cuPDLPx family -- but does not print its update,
restart rule, step size, weights or termination formula.  This module writes
those steps out from the LP and its optimality conditions (eq. (1), eq. (2))
and from the published PDHG method the paper cites; every constant is a field
of :class:`Opts`, the same fields the C ABI's ``lp_solve_opts`` carries.
Readings (choices where the paper is silent) are marked READING.

Pins (tests/test_oracle_pdhg.py): the planted optimum of every generator is a
fixed point of the operator T for any step sizes; vertex enumeration and
``scipy.optimize.linprog(method="highs")`` fix the optimal objective of tiny
and small LPs; with rho = 0 and no anchor the iteration reproduces a textbook
equality-form PDHG written independently; a 1 x 1 LP has a closed-form
solution; rel-KKT takes hand-computed values on 1-D examples; the power
iteration matches numpy's 2-norm (and finds the norm of matrices whose rows
sum to zero); scaling leaves a signed permutation matrix unchanged; the
infeasibility certificates accept hand-made Farkas rays and reject
near-misses, and LPs without an optimum get the status HiGHS reports; on an
LP whose operator T is constant (fixed columns, free rows) the iterates have
a closed form, which fixes the restart residual ||z - T(z)||_omega at every
check, the check at which criterion (i) and criterion (ii) each first fire,
and the primal weight after the restart for two values of theta (and its
band).  Feasibility polishing and the separate gap tolerance
(tests/test_oracle_polish.py): zeroing c leaves every primal residual and
zeroing the finite bounds every dual residual unchanged; the phases' points
are feasible by a direct evaluation of eq. (1) and of eq. (2)'s sign rules;
a polished solve meets the test with the objective HiGHS finds, within the
gap tolerance; failed attempts leave the main iterates bit for bit those of
a solve without polishing; the phase budget rounds up to a check period.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# termination codes (same numbering as the C ABI)
OPTIMAL, ITER_LIMIT, TIME_LIMIT, NUMERICAL, INFEASIBLE, UNBOUNDED = 0, 1, 2, 3, 4, 5


@dataclass
class Opts:
    eps_rel: float = 1e-6
    max_iter: int = 200_000
    time_limit_s: float = math.inf
    check_every: int = 64  # K, READING: restart/termination checks every 64 iterations
    rho: float = 1.0  # reflection, READING: 1 (r2HPDHG); rho = 0 is plain Halpern
    beta_suff: float = 0.2  # READING: PDLP's restart constants
    beta_nec: float = 0.8
    beta_art: float = 0.36
    theta: float = 0.5  # primal-weight smoothing
    omega_clamp: float = 10.0  # READING: omega kept within [omega0 / c, omega0 * c] (0: none)
    ruiz_iters: int = 10
    pock_chambolle: bool = True
    power_iters: int = 100
    halpern: bool = True  # False: plain PDHG z <- (1+rho)T(z) - rho z (no anchor)
    restarts: bool = True
    infeas_every: int = 4  # READING: infeasibility test every 4th check (0: never)
    eps_infeas: float = 1e-8  # READING: PDLP's infeasibility tolerances
    eps_gap: float | None = None  # relative gap tolerance (None: eps_rel; see pdhg_solve)
    polish: bool = False  # READING: feasibility polishing (see feasibility_polish), off
    polish_fraction: float = 0.125  # a polishing phase runs at most max(K, fraction * t) iterations


@dataclass
class Result:
    status: int
    x: np.ndarray  # T(z) at termination, unscaled
    y: np.ndarray
    z: np.ndarray  # c - A^T y, unscaled (reduced costs of the returned y)
    x_iter: np.ndarray  # current iterate z^t, unscaled
    y_iter: np.ndarray
    iterations: int
    restarts: int
    kkt: dict
    eta: float
    omega: float
    omega0: float
    iterates: list = field(default_factory=list)
    checks: list = field(default_factory=list)
    polish: dict = field(default_factory=dict)  # attempts, successes, phase iterations


# ----------------------------------------------------------------------------
# problem access


def csr_of(lp) -> sp.csr_matrix:
    return sp.csr_matrix(
        (np.asarray(lp.val, dtype=np.float64), np.asarray(lp.col_idx, dtype=np.int64),
         np.asarray(lp.row_ptr, dtype=np.int64)), shape=(lp.m, lp.n))


def box(v, lo, hi):
    """Euclidean projection onto [lo, hi] (componentwise, infinite ends allowed)."""
    return np.minimum(np.maximum(v, lo), hi)


# ----------------------------------------------------------------------------
# optimality measure (eq. (2))


def dual_cone_project(g, col_lo, col_hi):
    """Project g onto Lambda = prod_j Lambda_j, the sign set that eq. (2) allows
    for z_j: {0} for a free column, [0, inf) if only the lower bound is finite,
    (-inf, 0] if only the upper bound is finite, R if both are finite."""
    lf = np.isfinite(col_lo)
    uf = np.isfinite(col_hi)
    lam = np.array(g, dtype=np.float64, copy=True)
    lam[~lf & ~uf] = 0.0
    only_l = lf & ~uf
    only_u = ~lf & uf
    lam[only_l] = np.maximum(lam[only_l], 0.0)
    lam[only_u] = np.minimum(lam[only_u], 0.0)
    return lam


def dual_row_project(y, row_lo, row_hi):
    """Sign domain of y_i from eq. (2): y_i <= 0 if row_lo_i = -inf,
    y_i >= 0 if row_hi_i = +inf (so 0 if both are infinite)."""
    out = np.array(y, dtype=np.float64, copy=True)
    lf = np.isfinite(row_lo)
    uf = np.isfinite(row_hi)
    out[~lf] = np.minimum(out[~lf], 0.0)
    out[~uf] = np.maximum(out[~uf], 0.0)
    return out


def _support(v, lo, hi):
    """sum_i (v_i^+ lo_i - v_i^- hi_i) with 0 * inf := 0."""
    pos = v > 0
    neg = v < 0
    s = 0.0
    if pos.any():
        s += float(np.sum(v[pos] * lo[pos]))
    if neg.any():
        s += float(np.sum(v[neg] * hi[neg]))
    return s


def infeasibility_certificate(lp, A, d, w, eps):
    """Test a direction (d, w) of the iterates for a certificate that the LP
    of eq. (1) has no optimum (READING: the paper's solver family detects
    infeasibility from iterate differences; the tests are the Farkas
    alternatives of eq. (2) with relative tolerance eps).

    Primal infeasibility (dual ray): wp = w projected on the rows' sign
    domain, lam = proj_Lambda(-A^T wp); a certificate when the dual objective
    D = sum(wp^+ l_c - wp^- u_c) + sum(lam^+ l_x - lam^- u_x) > 0 and
    ||A^T wp + lam||_2 <= eps D (then every dual-feasible point can be moved
    along (wp, lam) with the dual objective growing without bound).

    Dual infeasibility (primal ray): c^T d < 0 and the violation of A d
    against the recession cone of [l_c, u_c] ((A d)_i <= 0 where u_ci is
    finite, >= 0 where l_ci is) together with that of d against the
    recession cone of [l_x, u_x], in 2-norm, is at most eps (-c^T d).

    A and all vectors in the problem's own (unscaled) units.  Returns
    INFEASIBLE, UNBOUNDED or None; the dual ray is tested first."""
    lo, hi = np.asarray(lp.row_lo, np.float64), np.asarray(lp.row_hi, np.float64)
    lx, ux = np.asarray(lp.col_lo, np.float64), np.asarray(lp.col_hi, np.float64)
    c = np.asarray(lp.c, np.float64)
    wp = dual_row_project(w, lo, hi)
    g = A.T @ wp
    lam = dual_cone_project(-g, lx, ux)
    dobj = _support(wp, lo, hi) + _support(lam, lx, ux)
    if dobj > 0 and float(np.linalg.norm(g + lam)) <= eps * dobj:
        return INFEASIBLE
    cd = float(c @ d)
    if cd < 0:
        ad = A @ d
        vr = (np.where(np.isfinite(hi), np.maximum(ad, 0.0), 0.0)
              + np.where(np.isfinite(lo), np.maximum(-ad, 0.0), 0.0))
        vc = (np.where(np.isfinite(ux), np.maximum(d, 0.0), 0.0)
              + np.where(np.isfinite(lx), np.maximum(-d, 0.0), 0.0))
        if math.sqrt(float(vr @ vr) + float(vc @ vc)) <= eps * (-cd):
            return UNBOUNDED
    return None


def bhat_norm(row_lo, row_hi):
    """2-norm of the finite entries of row_lo and row_hi, equality rows once."""
    lf = np.isfinite(row_lo)
    uf = np.isfinite(row_hi) & ~(lf & (row_lo == row_hi))
    return float(math.sqrt(np.sum(row_lo[lf] ** 2) + np.sum(row_hi[uf] ** 2)))


def rel_kkt(lp, x, y, A=None):
    """Relative KKT error of (x, y) for eq. (1), from the conditions of eq. (2).

    READING (the paper fixes only eps_rel, not the formula): PDLP-style relative
    measure
      r_p   = || A x - proj_[l_c,u_c](A x) ||_2
      lam   = proj_Lambda(c - A^T y)                      (sign rules of eq. (2))
      r_d   = || (c - A^T y - lam,  y - proj_Y(y)) ||_2    (y outside its sign
              domain counts as dual infeasibility; it never is for PDHG output)
      p     = c^T x + off
      d     = sum_i (yp_i^+ l_ci - yp_i^- u_ci) + sum_j (lam_j^+ l_xj - lam_j^- u_xj) + off,
              yp = proj_Y(y), 0 * inf := 0
      relKKT = max(r_p / (1 + ||bhat||), r_d / (1 + ||c||), |p - d| / (1 + |p| + |d|)).
    x is taken as given (PDHG output lies in the column bounds).
    """
    if A is None:
        A = csr_of(lp)
    c = np.asarray(lp.c, dtype=np.float64)
    lo, hi = np.asarray(lp.row_lo, np.float64), np.asarray(lp.row_hi, np.float64)
    lx, ux = np.asarray(lp.col_lo, np.float64), np.asarray(lp.col_hi, np.float64)
    ax = A @ x
    rp_vec = ax - box(ax, lo, hi)
    g = c - A.T @ y
    lam = dual_cone_project(g, lx, ux)
    yp = dual_row_project(y, lo, hi)
    r_p = float(np.linalg.norm(rp_vec))
    r_d = float(math.sqrt(np.sum((g - lam) ** 2) + np.sum((y - yp) ** 2)))
    p = float(c @ x) + float(lp.obj_offset)
    d = _support(yp, lo, hi) + _support(lam, lx, ux) + float(lp.obj_offset)
    nb = bhat_norm(lo, hi)
    nc = float(np.linalg.norm(c))
    rel_p = r_p / (1.0 + nb)
    rel_d = r_d / (1.0 + nc)
    gap = abs(p - d)
    rel_gap = gap / (1.0 + abs(p) + abs(d))
    return {"r_p": r_p, "r_d": r_d, "gap": gap, "p": p, "d": d, "rel_p": rel_p,
            "rel_d": rel_d, "rel_gap": rel_gap, "rel_kkt": max(rel_p, rel_d, rel_gap),
            "bhat_norm": nb, "c_norm": nc}


# ----------------------------------------------------------------------------
# preconditioning and step size (READING: the paper is silent)


def ruiz_pc_scaling(A: sp.csr_matrix, ruiz_iters: int = 10, pock_chambolle: bool = True):
    """Diagonal scalings D_r, D_c with scaled matrix D_r A D_c.

    READING: ``ruiz_iters`` Ruiz equilibration passes, each dividing every row
    and column of the current scaled matrix by the square root of its largest
    absolute entry (both computed from the same current matrix; empty rows and
    columns keep factor 1), then one Pock-Chambolle pass with alpha = 1
    dividing by the square root of the absolute row and column sums.
    """
    m, n = A.shape
    dr = np.ones(m)
    dc = np.ones(n)
    absA = abs(A).tocsr()
    for _ in range(ruiz_iters):
        S = sp.diags(dr) @ absA @ sp.diags(dc)
        rmax = np.asarray(S.max(axis=1).todense()).ravel()
        cmax = np.asarray(S.max(axis=0).todense()).ravel()
        rmax = np.where(rmax > 0, rmax, 1.0)
        cmax = np.where(cmax > 0, cmax, 1.0)
        dr = dr / np.sqrt(rmax)
        dc = dc / np.sqrt(cmax)
    if pock_chambolle:
        S = sp.diags(dr) @ absA @ sp.diags(dc)
        rsum = np.asarray(S.sum(axis=1)).ravel()
        csum = np.asarray(S.sum(axis=0)).ravel()
        rsum = np.where(rsum > 0, rsum, 1.0)
        csum = np.where(csum > 0, csum, 1.0)
        dr = dr / np.sqrt(rsum)
        dc = dc / np.sqrt(csum)
    return dr, dc


def power_norm(A: sp.spmatrix, iters: int = 100) -> float:
    """Estimate ||A||_2 by power iteration on A^T A.

    READING: start vector all-ones / sqrt(n); each step v <- A^T (A v) / ||.||;
    the estimate is ||A v||_2 for the final vector v.  A step that gives the
    zero vector (all-ones is orthogonal to every right singular vector with a
    nonzero value when the rows of A sum to zero, e.g. A = [1, -1]) continues
    from the fallback v_j = (0.5 + h(j) / 2^32) / sqrt(n), with the
    multiplicative hash h(j) = j * 2654435761 mod 2^32 of the column index.
    """
    m, n = A.shape
    if n == 0 or m == 0:
        return 0.0
    v = np.full(n, 1.0 / math.sqrt(n))
    h = (np.arange(n, dtype=np.uint64) * np.uint64(2654435761)) % np.uint64(2 ** 32)
    fallback = (0.5 + h.astype(np.float64) / 4294967296.0) * (1.0 / math.sqrt(n))
    for _ in range(iters):
        w = A.T @ (A @ v)
        nw = float(np.linalg.norm(w))
        v = w / nw if nw > 0.0 else fallback
    return float(np.linalg.norm(A @ v))


# ----------------------------------------------------------------------------
# the PDHG operator and the restarted Halpern iteration


def pdhg_operator(A, c, lx, ux, lc, uc, x, y, tau, sigma):
    """One PDHG step T(x, y) for the saddle problem of eq. (1):
      xh = proj_[lx,ux](x - tau (c - A^T y))
      xb = 2 xh - x
      v  = y - sigma A xb
      yh = v + sigma proj_[lc,uc](-v / sigma)   (prox of the row-bound conjugate)
    """
    xh = box(x - tau * (c - A.T @ y), lx, ux)
    xb = 2.0 * xh - x
    v = y - sigma * (A @ xb)
    yh = v + sigma * box(-v / sigma, lc, uc)
    return xh, yh


class Scaled:
    """The problem after scaling: A~ = D_r A D_c, c~ = D_c c, row bounds D_r l,
    column bounds l / D_c."""

    def __init__(self, lp, opts: Opts):
        A = csr_of(lp)
        self.A0 = A
        self.dr, self.dc = ruiz_pc_scaling(A, opts.ruiz_iters, opts.pock_chambolle)
        self.A = (sp.diags(self.dr) @ A @ sp.diags(self.dc)).tocsr()
        self.c = self.dc * np.asarray(lp.c, np.float64)
        self.lc = self.dr * np.asarray(lp.row_lo, np.float64)
        self.uc = self.dr * np.asarray(lp.row_hi, np.float64)
        self.lx = np.asarray(lp.col_lo, np.float64) / self.dc
        self.ux = np.asarray(lp.col_hi, np.float64) / self.dc


def default_omega(sc: Scaled) -> float:
    """READING: omega_0 = ||c~||_2 / ||bhat~||_2, 1 if either is 0."""
    nc = float(np.linalg.norm(sc.c))
    nb = bhat_norm(sc.lc, sc.uc)
    if nc > 0 and nb > 0:
        return nc / nb
    return 1.0


def pdhg_solve(lp, opts: Opts | None = None, eta: float | None = None,
               omega0: float | None = None, x_init=None, y_init=None,
               record_iterates: int = 0, record_checks: bool = False,
               check_lp=None, stop_on: str = "kkt") -> Result:
    """Restarted reflected Halpern PDHG (READING of the solver the paper times).

    State z = (x, y) in the scaled space, anchor z0, Halpern counter k.
    Iteration t = 0, 1, ...:
      1. (xh, yh) = T(z)                                   (pdhg_operator)
      2. if t % K == 0 (a check):
         a. stop if relKKT(unscaled xh, yh) <= eps_rel (return T(z)), or on
            non-finite values, or past the time limit; else, at every
            infeas_every-th check, stop with INFEASIBLE / UNBOUNDED when the
            direction T(z) - z0 (unscaled) passes infeasibility_certificate;
         b. r = ||z - T(z)||_omega,  ||(a, b)||_omega^2 = omega ||a||^2 + ||b||^2 / omega;
         c. k == 0 (t = 0): r0 = r_prev = r;
            else restart if (i) r <= beta_suff r0, or (ii) r <= beta_nec r0 and
            r > r_prev, or (iii) k >= beta_art t.  On restart: new anchor
            z0' = T(z); primal weight omega <- exp(theta log(dy/dx) +
            (1 - theta) log omega) with dx = ||x0' - x0||, dy = ||y0' - y0||
            when both exceed 1e-10, then kept within [omega0 / omega_clamp,
            omega0 * omega_clamp] (READING, omega_clamp = 10; a weight that
            drifts by orders of magnitude stalled some planted LPs for
            100k+ iterations); z = z0 = T(z); k = 0; r0 = r_prev = r;
            skip step 3.  Otherwise r_prev = r.
      3. z <- lam_k ((1 + rho) T(z) - rho z) + (1 - lam_k) z0,  lam_k = (k+1)/(k+2);
         k <- k + 1.   (halpern=False: z <- (1 + rho) T(z) - rho z.)
    tau = eta / omega, sigma = eta * omega; eta = 0.998 / ||A~||_2 unless given.
    Initial point (READING): x = proj_[lx~,ux~](0), y = 0, or the given warm start.

    The checks evaluate rel-KKT of `check_lp` (default: lp itself, which must
    have the same matrix).  stop_on="kkt" stops when rel_p <= eps_rel,
    rel_d <= eps_rel and rel_gap <= eps_gap (eps_gap = eps_rel unless set:
    then this is rel-KKT <= eps_rel); "primal" / "dual" stop on rel_p / rel_d
    alone (the phases of feasibility_polish).  With opts.polish, a check that
    does not stop and finds rel_gap <= eps_gap while max(rel_p, rel_d) >
    eps_rel, at t at or past the next allowed attempt, runs
    feasibility_polish from T(z); when the polished pair meets the stopping
    test the solve stops OPTIMAL with it, else the next attempt waits until
    t >= 2 t (READING).  `iterations` then also counts the phases'.
    """
    opts = opts or Opts()
    check_lp = lp if check_lp is None else check_lp
    sc = Scaled(lp, opts)
    A = sc.A
    m, n = A.shape
    if eta is None:
        nrm = power_norm(A, opts.power_iters)
        eta = 0.998 / nrm if nrm > 0 else 1.0
    if omega0 is None:
        omega0 = default_omega(sc)
    omega = float(omega0)
    if x_init is None:
        x = box(np.zeros(n), sc.lx, sc.ux)
    else:
        x = np.asarray(x_init, np.float64) / sc.dc
    y = np.zeros(m) if y_init is None else np.asarray(y_init, np.float64) / sc.dr
    x0, y0 = x.copy(), y.copy()
    K = max(int(opts.check_every), 1)
    k = 0
    t = 0
    restarts = 0
    r0 = r_prev = None
    status = ITER_LIMIT
    kkt = None
    xh = x
    yh = y
    iterates = []
    checks = []
    polish = {"attempts": 0, "successes": 0, "phase_iterations": 0}
    next_polish = 0
    polished = None
    start = time.perf_counter()
    if record_iterates:
        iterates.append((sc.dc * x, sc.dr * y))
    while t < opts.max_iter:
        tau = eta / omega
        sigma = eta * omega
        xh, yh = pdhg_operator(A, sc.c, sc.lx, sc.ux, sc.lc, sc.uc, x, y, tau, sigma)
        if t % K == 0:
            kkt = rel_kkt(check_lp, sc.dc * xh, sc.dr * yh, A=sc.A0)
            if stop_on == "kkt":
                done = kkt_met(kkt, opts)
            else:
                done = kkt["rel_p" if stop_on == "primal" else "rel_d"] <= opts.eps_rel
            if record_checks:
                checks.append({"t": t, "rel_kkt": kkt["rel_kkt"], "omega": omega, "k": k})
            if not (np.all(np.isfinite(xh)) and np.all(np.isfinite(yh))
                    and math.isfinite(kkt["rel_kkt"])):
                status = NUMERICAL
            elif done:
                status = OPTIMAL
            elif time.perf_counter() - start > opts.time_limit_s:
                status = TIME_LIMIT
            elif opts.infeas_every > 0 and (t // K) % opts.infeas_every == 0:
                # direction since the last restart: T(z) - z0, unscaled
                cert = infeasibility_certificate(lp, sc.A0, sc.dc * (xh - x0), sc.dr * (yh - y0),
                                                 opts.eps_infeas)
                if cert is not None:
                    status = cert
            if (status == ITER_LIMIT and opts.polish and stop_on == "kkt" and t >= next_polish
                    and kkt["rel_gap"] <= gap_tol(opts)
                    and max(kkt["rel_p"], kkt["rel_d"]) > opts.eps_rel):
                got = feasibility_polish(lp, opts, sc.dc * xh, sc.dr * yh, eta, omega, t)
                polish["attempts"] += 1
                polish["phase_iterations"] += got["iterations"]
                if got["kkt"] is not None and kkt_met(got["kkt"], opts):
                    polish["successes"] += 1
                    polished = got
                    status = OPTIMAL
                else:
                    next_polish = 2 * t
            if status != ITER_LIMIT:
                t += 1  # count this evaluation of T
                break
            r = math.sqrt(omega * float(np.sum((x - xh) ** 2))
                          + float(np.sum((y - yh) ** 2)) / omega)
            if record_checks:
                checks[-1]["r"] = r
            if k == 0:
                r0 = r_prev = r
            elif opts.restarts and (
                r <= opts.beta_suff * r0
                or (r <= opts.beta_nec * r0 and r > r_prev)
                or k >= opts.beta_art * t
            ):
                dx = float(np.linalg.norm(xh - x0))
                dy = float(np.linalg.norm(yh - y0))
                if dx > 1e-10 and dy > 1e-10:
                    omega = math.exp(opts.theta * math.log(dy / dx)
                                     + (1.0 - opts.theta) * math.log(omega))
                if opts.omega_clamp > 0:
                    omega = min(max(omega, omega0 / opts.omega_clamp), omega0 * opts.omega_clamp)
                x, y = xh.copy(), yh.copy()
                x0, y0 = xh.copy(), yh.copy()
                k = 0
                r0 = r_prev = r
                restarts += 1
                if record_checks:
                    checks[-1]["restart"] = True
                    checks[-1]["omega_after"] = omega
                t += 1
                if record_iterates and t <= record_iterates:
                    iterates.append((sc.dc * x, sc.dr * y))
                continue
            else:
                r_prev = r
        if opts.halpern:
            lam = (k + 1.0) / (k + 2.0)
            x = lam * ((1.0 + opts.rho) * xh - opts.rho * x) + (1.0 - lam) * x0
            y = lam * ((1.0 + opts.rho) * yh - opts.rho * y) + (1.0 - lam) * y0
        else:
            x = (1.0 + opts.rho) * xh - opts.rho * x
            y = (1.0 + opts.rho) * yh - opts.rho * y
        k += 1
        t += 1
        if record_iterates and t <= record_iterates:
            iterates.append((sc.dc * x, sc.dr * y))
    if kkt is None or status == ITER_LIMIT:
        kkt = rel_kkt(check_lp, sc.dc * xh, sc.dr * yh, A=sc.A0)
    xs = sc.dc * xh
    ys = sc.dr * yh
    if polished is not None:
        xs, ys, kkt = polished["x"], polished["y"], polished["kkt"]
    zs = np.asarray(lp.c, np.float64) - sc.A0.T @ ys
    return Result(status=status, x=xs, y=ys, z=zs, x_iter=sc.dc * x, y_iter=sc.dr * y,
                  iterations=t + polish["phase_iterations"], restarts=restarts, kkt=kkt,
                  eta=float(eta), omega=omega, omega0=float(omega0), iterates=iterates,
                  checks=checks, polish=polish)


def gap_tol(opts: Opts) -> float:
    return opts.eps_rel if opts.eps_gap is None else opts.eps_gap


def kkt_met(kkt: dict, opts: Opts) -> bool:
    """The stopping test: rel_p, rel_d <= eps_rel and rel_gap <= eps_gap."""
    return (kkt["rel_p"] <= opts.eps_rel and kkt["rel_d"] <= opts.eps_rel
            and kkt["rel_gap"] <= gap_tol(opts))


class _Modified:
    """lp with its cost vector and / or its finite bounds replaced (the same
    matrix, so the same scaling)."""

    def __init__(self, lp, zero_cost=False, zero_bounds=False):
        for a in ("m", "n", "row_ptr", "col_idx", "val"):
            setattr(self, a, getattr(lp, a))
        self.c = np.zeros(lp.n) if zero_cost else np.asarray(lp.c, np.float64)
        self.obj_offset = 0.0 if zero_cost else float(lp.obj_offset)

        def z(v):
            v = np.asarray(v, np.float64)
            return np.where(np.isfinite(v), 0.0, v) if zero_bounds else v

        self.row_lo, self.row_hi = z(lp.row_lo), z(lp.row_hi)
        self.col_lo, self.col_hi = z(lp.col_lo), z(lp.col_hi)


def feasibility_polish(lp, opts: Opts, x_hat, y_hat, eta: float, omega: float, t: int) -> dict:
    """Feasibility polishing (READING; the PDLP family's variant, which the
    paper does not specify).  From a point whose duality gap already meets
    eps_rel, two PDHG runs on feasibility problems of the same matrix:
      primal phase: the LP with c = 0 (any feasible x is optimal), from
        (x_hat, 0), stopped when rel_p of the ORIGINAL LP is <= eps_rel;
      dual phase: the LP with every finite bound set to 0 (its dual has the
        same feasible set as the original's, with objective 0), from
        (0, y_hat), stopped when rel_d of the original LP is <= eps_rel;
    each a fresh restarted Halpern PDHG (same options, no infeasibility test,
    no polishing) with the solve's eta and omega_0 = the current omega, at
    most max(K, polish_fraction * t) iterations rounded up to a multiple of
    K.  The candidate is (x of the primal phase, y of the dual phase): both
    moved little from (x_hat, y_hat), so their gap stays near the gap of
    (x_hat, y_hat); the caller accepts it when it meets the stopping test
    (kkt_met) on the original LP.  The phases stay near (x_hat, y_hat) in
    norm, but the gap of the pair grows with the moves (measured: 2e-4 to
    1e-3 relative from points at 1e-5 feasibility), so polishing pays only
    with eps_gap well above eps_rel, the regime it is meant for.
    Returns {"x", "y", "kkt" (None if a phase failed), "iterations"}.
    """
    K = max(int(opts.check_every), 1)
    budget = K * max(1, math.ceil(opts.polish_fraction * t / K))
    sub = Opts(**{**opts.__dict__, "max_iter": budget, "infeas_every": 0, "polish": False})
    rp = pdhg_solve(_Modified(lp, zero_cost=True), sub, eta=eta, omega0=omega,
                    x_init=x_hat, y_init=np.zeros(lp.m), check_lp=lp, stop_on="primal")
    out = {"x": None, "y": None, "kkt": None, "iterations": rp.iterations}
    if rp.status != OPTIMAL:
        return out
    rd = pdhg_solve(_Modified(lp, zero_bounds=True), sub, eta=eta, omega0=omega,
                    x_init=np.zeros(lp.n), y_init=y_hat, check_lp=lp, stop_on="dual")
    out["iterations"] += rd.iterations
    if rd.status != OPTIMAL:
        return out
    out["x"], out["y"] = rp.x, rd.y
    out["kkt"] = rel_kkt(lp, rp.x, rd.y)
    return out
