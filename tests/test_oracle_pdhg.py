"""Pins for the oracle PDHG (CPU only).

Each pin ties the oracle to something other than itself: the planted optimum
(fixed by construction through eq. (2)), vertex enumeration, scipy's HiGHS,
hand-computed values, numpy's matrix 2-norm, or a textbook equality-form PDHG
written here independently of the oracle's general prox form.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
from oracle import pdhg as P
from oracle.vertex import vertex_optimum
from lp_helpers import SimpleLP, highs_solve


def rel_obj_err(p, q):
    return abs(p - q) / (1.0 + abs(q))


# ---------------------------------------------------------------------------
# the planted optimum is a fixed point of T for any step sizes


@pytest.mark.parametrize("make", [
    lambda: lpgen.c1_small(),
    lambda: lpgen.general_structure(300, 700, 11, nnz_target=4000, one_sided=0.3),
    lambda: lpgen.c3_powerlaw(seed=5, m=400, n=1000, row_nnz_target=6000, n_dense=5,
                              dense_len=60),
    lambda: lpgen.tiny_box(4, 6, 3),
])
def test_planted_point_is_fixed_point(make):
    lp = make()
    sc = P.Scaled(lp, P.Opts())
    xs, ys = lp.x_star / sc.dc, lp.y_star / sc.dr
    rng = np.random.default_rng(0)
    for _ in range(3):
        tau, sigma = rng.uniform(0.01, 2.0, size=2)
        xh, yh = P.pdhg_operator(sc.A, sc.c, sc.lx, sc.ux, sc.lc, sc.uc, xs, ys, tau, sigma)
        assert np.max(np.abs(xh - xs)) <= 1e-9 * (1 + np.max(np.abs(xs)))
        assert np.max(np.abs(yh - ys)) <= 1e-9 * (1 + np.max(np.abs(ys)))
    k = oracle.rel_kkt(lp, lp.x_star, lp.y_star)
    assert k["rel_kkt"] <= 1e-12


def test_planted_point_moves_when_perturbed():
    # a non-optimal point is not a fixed point (guards against a T that is the identity)
    lp = lpgen.c1_small()
    sc = P.Scaled(lp, P.Opts())
    xs, ys = lp.x_star / sc.dc + 0.01, lp.y_star / sc.dr
    xh, yh = P.pdhg_operator(sc.A, sc.c, sc.lx, sc.ux, sc.lc, sc.uc, xs, ys, 0.5, 0.5)
    assert np.max(np.abs(xh - xs)) + np.max(np.abs(yh - ys)) > 1e-4


# ---------------------------------------------------------------------------
# vertex enumeration and HiGHS fix the objective


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_vertex_enumeration_agrees_with_highs_and_plant(seed):
    lp = lpgen.tiny_box(4, 5, seed)
    pv, _ = vertex_optimum(lp)
    ph, _, _ = highs_solve(lp)
    assert abs(pv - ph) <= 1e-9 * (1 + abs(ph))
    assert abs(pv - lp.p_star) <= 1e-9 * (1 + abs(pv))


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_pdhg_reaches_vertex_optimum(seed):
    lp = lpgen.tiny_box(4, 5, seed)
    pv, _ = vertex_optimum(lp)
    r = oracle.pdhg_solve(lp, P.Opts(eps_rel=1e-8))
    assert r.status == P.OPTIMAL
    assert r.kkt["rel_kkt"] <= 1e-8
    assert rel_obj_err(r.kkt["p"], pv) <= 1e-6


def test_c1_converges_to_planted_optimum():
    lp = lpgen.c1_small()
    ph, _, _ = highs_solve(lp)
    assert rel_obj_err(ph, lp.p_star) <= 1e-9
    r = oracle.pdhg_solve(lp)
    assert r.status == P.OPTIMAL
    assert r.kkt["rel_kkt"] <= 1e-6
    assert rel_obj_err(r.kkt["p"], lp.p_star) <= 1e-6
    assert r.restarts >= 1


def test_small_presolvable_structure_converges():
    lp = lpgen.general_structure(400, 1000, 21, nnz_target=8000, one_sided=0.2)
    ph, _, _ = highs_solve(lp)
    assert rel_obj_err(ph, lp.p_star) <= 1e-8
    r = oracle.pdhg_solve(lp)
    assert r.status == P.OPTIMAL
    assert rel_obj_err(r.kkt["p"], lp.p_star) <= 1e-5


# ---------------------------------------------------------------------------
# special cases that reduce to a textbook method


def _textbook_equality_pdhg(A, b, c, tau, sigma, iters, halpern, rho):
    """Textbook PDHG for min c^T x, A x = b, x >= 0 (dense, no scaling):
    x+ = max(0, x - tau (c - A^T y)),  y+ = y + sigma (b - A (2 x+ - x));
    optionally reflected (rho) and Halpern-anchored at the start point."""
    m, n = A.shape
    x = np.zeros(n)
    y = np.zeros(m)
    x0, y0 = x.copy(), y.copy()
    out = []
    for k in range(iters):
        xp = np.maximum(0.0, x - tau * (c - A.T @ y))
        yp = y + sigma * (b - A @ (2 * xp - x))
        rx, ry = (1 + rho) * xp - rho * x, (1 + rho) * yp - rho * y
        if halpern:
            w = (k + 1) / (k + 2)
            x, y = w * rx + (1 - w) * x0, w * ry + (1 - w) * y0
        else:
            x, y = rx, ry
        out.append((x.copy(), y.copy()))
    return out


@pytest.mark.parametrize("halpern,rho", [(False, 0.0), (True, 0.0), (True, 1.0), (True, 0.5)])
def test_matches_textbook_equality_pdhg(halpern, rho):
    lp = lpgen.equality_nonneg(30, 60, 5, 3, 8)
    A = lp.csr().toarray()
    b = lp.row_lo.copy()
    opts = P.Opts(max_iter=40, check_every=10_000, ruiz_iters=0, pock_chambolle=False,
                  halpern=halpern, rho=rho, restarts=False)
    eta, omega = 0.9 / np.linalg.norm(A, 2), 1.7
    r = oracle.pdhg_solve(lp, opts, eta=eta, omega0=omega, record_iterates=40)
    ref = _textbook_equality_pdhg(A, b, lp.c, eta / omega, eta * omega, 40, halpern, rho)
    for k in range(40):
        xo, yo = r.iterates[k + 1]
        xr, yr = ref[k]
        assert np.allclose(xo, xr, rtol=1e-12, atol=1e-12)
        assert np.allclose(yo, yr, rtol=1e-12, atol=1e-12)


def test_matches_textbook_inequality_pdhg():
    # A x >= b, x >= 0: textbook y+ = max(0, y + sigma (b - A xbar))
    rng = np.random.default_rng(3)
    A = rng.standard_normal((12, 20))
    b = rng.standard_normal(12)
    c = np.abs(rng.standard_normal(20))
    lp = SimpleLP(A, c, b, np.full(12, np.inf), np.zeros(20), np.full(20, np.inf))
    opts = P.Opts(max_iter=30, check_every=10_000, ruiz_iters=0, pock_chambolle=False,
                  halpern=False, rho=0.0, restarts=False)
    tau, sigma = 0.05, 0.08
    eta, omega = math.sqrt(tau * sigma), math.sqrt(sigma / tau)
    r = oracle.pdhg_solve(lp, opts, eta=eta, omega0=omega, record_iterates=30)
    x = np.zeros(20)
    y = np.zeros(12)
    for k in range(30):
        xp = np.maximum(0, x - tau * (c - A.T @ y))
        y = np.maximum(0, y + sigma * (b - A @ (2 * xp - x)))
        x = xp
        xo, yo = r.iterates[k + 1]
        assert np.allclose(xo, x, atol=1e-11)
        assert np.allclose(yo, y, atol=1e-11)


def test_one_by_one_closed_form():
    # min -3 x  s.t. 1 <= 2 x <= 5, 0 <= x <= 2: optimum x = min(2, 5/2) = 2, p = -6;
    # the row is inactive at x = 2 (2x = 4 < 5) so y = 0 and z = c = -3 (upper bound).
    lp = SimpleLP([[2.0]], [-3.0], [1.0], [5.0], [0.0], [2.0])
    r = oracle.pdhg_solve(lp, P.Opts(eps_rel=1e-10))
    assert r.status == P.OPTIMAL
    assert abs(r.x[0] - 2.0) <= 1e-8
    assert abs(r.kkt["p"] + 6.0) <= 1e-8
    # tighten the row: 2 x <= 3 -> x = 1.5, y = c / a = -1.5, z = 0
    lp = SimpleLP([[2.0]], [-3.0], [1.0], [3.0], [0.0], [2.0])
    r = oracle.pdhg_solve(lp, P.Opts(eps_rel=1e-10))
    assert abs(r.x[0] - 1.5) <= 1e-8 and abs(r.y[0] + 1.5) <= 1e-8
    assert abs(r.kkt["p"] + 4.5) <= 1e-8


def test_first_check_restarts_and_resets_to_T():
    # criterion (iii) holds at the first check after t = 0 (k = t); after 65
    # evaluations of T the state is T(z^64), i.e. the anchor
    lp = lpgen.c1_small()
    r = oracle.pdhg_solve(lp, P.Opts(max_iter=65, eps_rel=0.0))
    assert r.restarts == 1
    r64 = oracle.pdhg_solve(lp, P.Opts(max_iter=65, eps_rel=0.0, restarts=False))
    # T(z^64) is the returned x of the no-restart run (last T evaluated)
    assert np.allclose(r.x_iter, r64.x, atol=1e-13)
    assert np.allclose(r.y_iter, r64.y, atol=1e-13)


# ---------------------------------------------------------------------------
# rel-KKT on hand-computed examples


def test_rel_kkt_hand_values():
    # min 2x  s.t. 1 <= x <= 3, 0 <= x <= 10, at x = 0.5, y = 1:
    # Ax = 0.5 -> r_p = 0.5; c - A^T y = 1, column boxed -> lam = 1, r_d = 0;
    # p = 1, d = y*1 + lam*0 = 1; ||bhat|| = sqrt(1 + 9).
    lp = SimpleLP([[1.0]], [2.0], [1.0], [3.0], [0.0], [10.0])
    k = oracle.rel_kkt(lp, np.array([0.5]), np.array([1.0]))
    assert k["r_p"] == 0.5 and k["r_d"] == 0.0
    assert k["p"] == 1.0 and k["d"] == 1.0
    assert abs(k["rel_p"] - 0.12012653667602105) < 1e-15
    assert abs(k["rel_kkt"] - 0.12012653667602105) < 1e-15
    # free column: lam = 0, r_d = |c - a y| = |2 - 3| = 1; y = 3 on a row with
    # l = 1: d = 3, p = 2 * 2 = 4 at x = 2 (feasible), gap 1 / (1 + 4 + 3)
    lp = SimpleLP([[1.0]], [2.0], [1.0], [3.0], [-np.inf], [np.inf])
    k = oracle.rel_kkt(lp, np.array([2.0]), np.array([3.0]))
    assert k["r_p"] == 0.0 and k["r_d"] == 1.0
    assert k["p"] == 4.0 and k["d"] == 3.0
    assert abs(k["rel_d"] - 1.0 / 3.0) < 1e-15
    assert abs(k["rel_gap"] - 0.125) < 1e-15
    # row with only a lower side: y must be >= 0; y = -2 is out of its domain
    # (counts 2 in r_d, and yp = 0 in d); x >= 0 column: c - A^T y = 1 - (-2) = 3 >= 0
    lp = SimpleLP([[1.0]], [1.0], [1.0], [np.inf], [0.0], [np.inf])
    k = oracle.rel_kkt(lp, np.array([1.0]), np.array([-2.0]))
    assert k["r_d"] == 2.0
    assert k["d"] == 0.0 and k["p"] == 1.0


# ---------------------------------------------------------------------------
# step size and scaling


def test_power_norm_matches_numpy():
    rng = np.random.default_rng(1)
    Q1, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    Q2, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    s = np.concatenate([[7.0, 2.0, 1.5], np.linspace(1.0, 0.1, 27)])
    M = Q1[:, :30] @ np.diag(s) @ Q2.T
    est = P.power_norm(sp.csr_matrix(M), 100)
    assert abs(est - np.linalg.norm(M, 2)) <= 1e-12 * 7
    A = lpgen.c1_small().csr()
    est = P.power_norm(A, 100)
    true = np.linalg.norm(A.toarray(), 2)
    assert est <= true * (1 + 1e-12)
    assert est >= true * 0.98


def test_scaling_leaves_signed_permutation_unchanged():
    rng = np.random.default_rng(2)
    p = rng.permutation(25)
    M = sp.csr_matrix((np.where(rng.random(25) < 0.5, -1.0, 1.0), (np.arange(25), p)),
                      shape=(25, 25))
    dr, dc = P.ruiz_pc_scaling(M, 10, True)
    assert np.all(dr == 1.0) and np.all(dc == 1.0)


def test_ruiz_equilibrates():
    A = lpgen.general_structure(200, 500, 3, nnz_target=3000).csr()
    dr, dc = P.ruiz_pc_scaling(A, 40, False)
    S = abs(sp.diags(dr) @ A @ sp.diags(dc)).tocsr()
    rmax = np.asarray(S.max(axis=1).todense()).ravel()
    cmax = np.asarray(S.max(axis=0).todense()).ravel()
    rmax = rmax[np.diff(A.indptr) > 0]
    cmax = cmax[np.diff(A.tocsc().indptr) > 0]
    assert np.all(np.abs(rmax - 1) < 1e-3) and np.all(np.abs(cmax - 1) < 1e-3)


def test_artificial_restart_schedule_hand_derived():
    # with criteria (i) and (ii) disabled, restarts happen at the checks
    # t = 64 j where the Halpern count k since the last restart satisfies
    # k >= 0.36 t: t = 64 (k = 64), 128 (63 >= 46.08), 256 (127 >= 92.16),
    # 448 (191 >= 161.28), 704 (255 >= 253.44)
    lp = lpgen.c1_small()
    opts = P.Opts(max_iter=1000, eps_rel=0.0, beta_suff=0.0, beta_nec=0.0)
    r = oracle.pdhg_solve(lp, opts, record_checks=True)
    ks = {c["t"]: c["k"] for c in r.checks}
    restarted = [t for t in sorted(ks) if t + 64 in ks and ks[t + 64] == 63]
    assert restarted == [64, 128, 256, 448, 704]
    assert r.restarts == 5


def test_scaling_closed_form_one_row():
    # A = [1, 3], one Ruiz pass then Pock-Chambolle (alpha = 1), by hand:
    # Ruiz: row max 3 -> dr = 1/sqrt(3); column maxes 1, 3 -> dc = (1, 1/sqrt(3));
    # scaled row (1/sqrt(3), 1); PC: row sum 1 + 1/sqrt(3), column sums
    # 1/sqrt(3) and 1 -> dr /= sqrt(1 + 1/sqrt(3)), dc = (3^(1/4), 1/sqrt(3)).
    A = sp.csr_matrix(np.array([[1.0, 3.0]]))
    dr, dc = P.ruiz_pc_scaling(A, 1, True)
    s3 = math.sqrt(3.0)
    assert abs(dr[0] - (1 / s3) / math.sqrt(1 + 1 / s3)) <= 1e-15
    assert abs(dc[0] - 3.0 ** 0.25) <= 1e-15
    assert abs(dc[1] - 1 / s3) <= 1e-15


def test_power_norm_of_rows_summing_to_zero():
    # A = [1, -1] has A 1 = 0: an all-ones start would stall at 0; the hashed
    # start finds ||A|| = sqrt(2) (and a graph incidence matrix its norm)
    assert abs(P.power_norm(sp.csr_matrix(np.array([[1.0, -1.0]])), 100) - np.sqrt(2.0)) <= 1e-14
    # incidence matrix of a directed cycle: every row sums to zero
    k = 7
    M = np.zeros((k, k))
    for e in range(k):
        M[e, e], M[(e + 1) % k, e] = 1.0, -1.0
    est = P.power_norm(sp.csr_matrix(M), 200)
    assert abs(est - np.linalg.norm(M, 2)) <= 1e-9


# ---------------------------------------------------------------------------
# infeasibility / unboundedness detection

from infeasible_lps import CASES as NO_OPTIMUM  # noqa: E402


def _highs_status(lp):
    from scipy.optimize import linprog

    A = lp.csr()
    lo, hi = np.asarray(lp.row_lo), np.asarray(lp.row_hi)
    eq = np.isfinite(lo) & np.isfinite(hi) & (lo == hi)
    up = np.isfinite(hi) & ~eq
    dn = np.isfinite(lo) & ~eq
    kw = {}
    if up.any() or dn.any():
        kw.update(A_ub=sp.vstack([A[up], -A[dn]]), b_ub=np.concatenate([hi[up], -lo[dn]]))
    if eq.any():
        kw.update(A_eq=A[eq], b_eq=lo[eq])
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lp.col_lo, lp.col_hi)]
    return linprog(lp.c, bounds=bounds, method="highs", **kw).status


@pytest.mark.parametrize("name,make,status", NO_OPTIMUM)
def test_detects_infeasible_and_unbounded_like_highs(name, make, status):
    lp = make()
    # HiGHS: 2 infeasible, 3 unbounded
    assert _highs_status(lp) == {4: 2, 5: 3}[status]
    r = oracle.pdhg_solve(lp, oracle.Opts(max_iter=20000))
    assert r.status == status, (name, r.status, r.iterations)


def test_certificate_tests_on_hand_made_rays():
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, -1.0]]))
    lp = SimpleLP(A.toarray(), [1.0, 1.0], [-np.inf, -2.0], [-1.0, 2.0], [0.0, 0.0],
                  [np.inf, np.inf])
    # Farkas: w = (-1, 0) (row 0 has only u_0 = -1, so w_0 <= 0 is allowed)
    # gives A^T w = (-1, -1), cancelled by lam = (1, 1) >= 0 on x >= 0, and
    # the dual objective -w_0^- u_0 = -(1)(-1) = 1 > 0
    assert P.infeasibility_certificate(lp, A, np.zeros(2), np.array([-1.0, 0.0]), 1e-8) == P.INFEASIBLE
    # the wrong sign is no certificate (and is projected away)
    assert P.infeasibility_certificate(lp, A, np.zeros(2), np.array([1.0, 0.0]), 1e-8) is None
    A = sp.csr_matrix(np.array([[1.0, -1.0]]))
    lp = SimpleLP(A.toarray(), [-1.0, -1.0], [-1.0], [1.0], [0.0, 0.0], [np.inf, np.inf])
    assert P.infeasibility_certificate(lp, A, np.array([1.0, 1.0]), np.zeros(1), 1e-8) == P.UNBOUNDED
    # (1, 0) lowers the cost but leaves the ranged row: no certificate
    assert P.infeasibility_certificate(lp, A, np.array([1.0, 0.0]), np.zeros(1), 1e-8) is None
    # (-1, -1) leaves x >= 0
    assert P.infeasibility_certificate(lp, A, np.array([-1.0, -1.0]), np.zeros(1), 1e-8) is None


def test_feasible_lps_are_never_flagged():
    for s in range(4):
        lp = lpgen.general_structure(300, 700, 100 + s, nnz_target=4000, one_sided=0.3)
        r = oracle.pdhg_solve(lp, oracle.Opts(max_iter=50000, infeas_every=1))
        assert r.status == P.OPTIMAL


def test_primal_weight_stays_in_its_band():
    # item 236 of the C4 batch: unbounded weight updates drift omega down by
    # 400x and the solve needs 138k iterations; kept within 10x of omega_0 it
    # reaches 1e-6 in under 3k (the band is the READING of the update)
    lp = lpgen.c4_batch(count=1, first=236)[0]
    r = oracle.pdhg_solve(lp, oracle.Opts(max_iter=6000), record_checks=True)
    w0 = r.omega0
    assert all(w0 / 10 * (1 - 1e-12) <= c["omega"] <= w0 * 10 * (1 + 1e-12) for c in r.checks)
    assert r.status == P.OPTIMAL and r.iterations < 6000
    free = oracle.pdhg_solve(lp, oracle.Opts(max_iter=6000, omega_clamp=0.0), record_checks=True)
    assert min(c["omega"] for c in free.checks) < w0 / 10  # the band was needed


# ---------------------------------------------------------------------------
# restart criteria (i), (ii) and the primal-weight update, on an LP whose
# operator T is constant, so every iterate has a closed form
#
# Two fixed columns (l = u = 0) and two free rows (l = -inf, u = +inf), no
# scaling.  Whatever z = (x, y) is, T(z) = (0, 0): x^ = proj_[0,0](.) = 0,
# and for a free row y^ = v + sigma proj_R(-v / sigma) = 0.  With omega_0 = 16
# and eta = 1/16 (tau = 1/256, sigma = 1) both are exact in floating point.
# Start at x = u0 with ||u0|| = 3 and y = w0 with ||w0|| = 12, so
# d_k = z_k - T(z_k) = z_k and R = ||d_0||_omega = sqrt(16 * 9 + 144 / 16)
# = sqrt(153).
#
# Halpern, rho = 0:  z_{k+1} = lam_k z* + (1 - lam_k) z_0  =>  d_k = d_0 / (k + 1).
# Halpern, rho = 1:  d_{k+1} = -lam_k d_k + (1 - lam_k) d_0  =>  d_1 = 0,
#                    d_2 = d_0 / 3, d_3 = 0, d_4 = d_0 / 5, ...
# On a restart at T(z) = z* the primal weight moves with dx = ||x^ - x0|| = 3,
# dy = ||y^ - y0|| = 12: omega = (dy / dx)^theta * omega_prev^(1 - theta).

_U0 = np.array([3 * 0.6, 3 * 0.8])
_W0 = np.array([12 * 0.6, -12 * 0.8])
_R = math.sqrt(153.0)


def _constant_T_lp():
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    inf = np.inf
    return SimpleLP(A, [1.0, -2.0], [-inf, -inf], [inf, inf], [0.0, 0.0], [0.0, 0.0])


def _constant_T_run(rho, K, beta_suff, beta_nec, max_iter, theta=0.25):
    opts = P.Opts(eps_rel=-1.0, max_iter=max_iter, check_every=K, rho=rho, beta_suff=beta_suff,
                  beta_nec=beta_nec, beta_art=2.0, theta=theta, ruiz_iters=0,
                  pock_chambolle=False, infeas_every=0)
    return oracle.pdhg_solve(_constant_T_lp(), opts, eta=1.0 / 16.0, omega0=16.0,
                             x_init=_U0, y_init=_W0, record_checks=True)


def test_restart_criterion_sufficient_decay_hand_derived():
    # rho = 0, checks at t = 0, 2, 4: r = R, R / 3, R / 5.  (ii) and (iii) are
    # off (beta_nec < 0, beta_art = 2 > k / t).  (i) r <= 0.21 r0 first holds
    # at k = 4 (1/5 <= 0.21 < 1/3).
    r = _constant_T_run(rho=0.0, K=2, beta_suff=0.21, beta_nec=-1.0, max_iter=5)
    ch = {c["t"]: c for c in r.checks}
    assert sorted(ch) == [0, 2, 4]
    for t, div in ((0, 1), (2, 3), (4, 5)):
        assert abs(ch[t]["r"] - _R / div) <= 1e-14 * _R, (t, ch[t]["r"])
    assert not ch[0].get("restart") and not ch[2].get("restart")
    assert ch[4].get("restart") and r.restarts == 1
    # just above the threshold (0.19 < 1/5) the check at t = 4 does not restart
    r = _constant_T_run(rho=0.0, K=2, beta_suff=0.19, beta_nec=-1.0, max_iter=5)
    assert r.restarts == 0


def test_restart_criterion_necessary_decay_and_growth_hand_derived():
    # rho = 1, a check every iteration: r = R, 0, R / 3, 0, R / 5.  (i) is off
    # (beta_suff < 0) until r0 becomes 0 after the first restart.
    # beta_nec = 0.8: at t = 1 r = 0 does not exceed r_prev = R; at t = 2
    # r = R / 3 <= 0.8 R and R / 3 > r_prev = 0: restart.
    r = _constant_T_run(rho=1.0, K=1, beta_suff=-1.0, beta_nec=0.8, max_iter=3)
    ch = {c["t"]: c for c in r.checks}
    assert abs(ch[0]["r"] - _R) <= 1e-14 * _R
    assert ch[1]["r"] == 0.0 and not ch[1].get("restart")
    assert abs(ch[2]["r"] - _R / 3) <= 1e-14 * _R and ch[2].get("restart")
    assert r.restarts == 1
    # beta_nec = 0.3: R / 3 > 0.3 R keeps t = 2 going; t = 3 has r ~ 0 < r_prev;
    # t = 4 has r = R / 5 <= 0.3 R and R / 5 > r_prev: the first restart is at t = 4
    r = _constant_T_run(rho=1.0, K=1, beta_suff=-1.0, beta_nec=0.3, max_iter=5)
    ch = {c["t"]: c for c in r.checks}
    assert [t for t in sorted(ch) if ch[t].get("restart")] == [4]
    assert abs(ch[4]["r"] - _R / 5) <= 1e-14 * _R


def test_primal_weight_update_hand_derived():
    # the restart of the test above at t = 2, with dx = 3, dy = 12, omega = 16:
    # theta = 1/4: (12/3)^(1/4) * 16^(3/4) = sqrt(2) * 8
    r = _constant_T_run(rho=1.0, K=1, beta_suff=-1.0, beta_nec=0.8, max_iter=3, theta=0.25)
    assert abs(r.omega - 8.0 * math.sqrt(2.0)) <= 1e-13
    # theta = 3/4: 4^(3/4) * 16^(1/4) = 2 sqrt(2) * 2
    r = _constant_T_run(rho=1.0, K=1, beta_suff=-1.0, beta_nec=0.8, max_iter=3, theta=0.75)
    assert abs(r.omega - 4.0 * math.sqrt(2.0)) <= 1e-13
    # no restart yet: the weight is still omega_0
    r = _constant_T_run(rho=1.0, K=1, beta_suff=-1.0, beta_nec=0.8, max_iter=2)
    assert r.omega == 16.0 and r.restarts == 0


def test_primal_weight_band_clamps_the_update():
    # dy / dx = 12 / 3e-6 = 4e6: (4e6)^(1/4) * 8 = 357.8 > 10 * omega_0 = 160
    lp = _constant_T_lp()
    opts = P.Opts(eps_rel=-1.0, max_iter=3, check_every=1, rho=1.0, beta_suff=-1.0,
                  beta_nec=0.8, beta_art=2.0, theta=0.25, ruiz_iters=0, pock_chambolle=False,
                  infeas_every=0)
    r = oracle.pdhg_solve(lp, opts, eta=1.0 / 16.0, omega0=16.0, x_init=_U0 * 1e-6, y_init=_W0)
    assert r.restarts == 1 and r.omega == 160.0
    opts.omega_clamp = 0.0
    r = oracle.pdhg_solve(lp, opts, eta=1.0 / 16.0, omega0=16.0, x_init=_U0 * 1e-6, y_init=_W0)
    assert abs(r.omega - 8.0 * (4e6) ** 0.25) <= 1e-9 * r.omega
