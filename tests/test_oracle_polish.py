"""Pins of the oracle's feasibility polishing and separate gap tolerance
(oracle/pdhg.py: feasibility_polish, kkt_met), checked against direct
evaluations of eq. (1) / eq. (2) and against HiGHS, not against the oracle's
own rel-KKT routine."""
import numpy as np

import lpgen
from oracle import pdhg as P
from lp_helpers import csr, highs_solve


def polish_lp():
    # a general-structure LP on which polishing succeeds at eps 1e-8 with a
    # gap tolerance of 1e-4 (measured: 8,705 plain iterations, 3,715 with it)
    return lpgen.general_structure(2000, 5000, 8, nnz_target=40_000, one_sided=0.2)


def mid_point(lp, iters):
    r = P.pdhg_solve(lp, P.Opts(eps_rel=0.0, max_iter=iters))
    return r


def primal_violation(lp, x):
    """|| A x - proj_[l_c, u_c](A x) ||_2 and the column-bound violation,
    written out from eq. (1)."""
    ax = csr(lp) @ x
    lo, hi = np.asarray(lp.row_lo, float), np.asarray(lp.row_hi, float)
    rv = np.maximum(lo - ax, 0.0) + np.maximum(ax - hi, 0.0)
    lx, ux = np.asarray(lp.col_lo, float), np.asarray(lp.col_hi, float)
    cv = np.maximum(lx - x, 0.0) + np.maximum(x - ux, 0.0)
    return float(np.linalg.norm(rv)), float(np.max(cv, initial=0.0))


def dual_violation(lp, y):
    """The violation of eq. (2)'s sign rules by y: reduced costs g = c - A^T y
    must be >= 0 on columns with only a finite lower bound, <= 0 with only a
    finite upper bound, 0 on free columns (any sign when both are finite);
    y_i >= 0 on rows with only a finite lower bound, <= 0 with only an upper
    one, 0 on free rows."""
    g = np.asarray(lp.c, float) - csr(lp).T @ y
    lx, ux = np.asarray(lp.col_lo, float), np.asarray(lp.col_hi, float)
    lf, uf = np.isfinite(lx), np.isfinite(ux)
    v = np.where(lf & ~uf, np.minimum(g, 0.0), 0.0)
    v += np.where(~lf & uf, np.maximum(g, 0.0), 0.0)
    v += np.where(~lf & ~uf, g, 0.0)
    lo, hi = np.asarray(lp.row_lo, float), np.asarray(lp.row_hi, float)
    rl, ru = np.isfinite(lo), np.isfinite(hi)
    w = np.where(rl & ~ru, np.minimum(y, 0.0), 0.0)
    w += np.where(~rl & ru, np.maximum(y, 0.0), 0.0)
    w += np.where(~rl & ~ru, y, 0.0)
    return float(np.sqrt(np.sum(v ** 2) + np.sum(w ** 2)))


def test_feasibility_problems_keep_the_measures_they_are_judged_by():
    # zeroing c leaves every primal residual alone; zeroing the finite bounds
    # leaves every dual residual alone (the dual sign rules depend only on
    # which bounds are finite): for any point, bit for bit
    lp = polish_lp()
    rng = np.random.default_rng(3)
    for _ in range(3):
        x = rng.normal(size=lp.n)
        y = rng.normal(size=lp.m)
        k0 = P.rel_kkt(lp, x, y)
        kc = P.rel_kkt(P._Modified(lp, zero_cost=True), x, y)
        kb = P.rel_kkt(P._Modified(lp, zero_bounds=True), x, y)
        assert kc["r_p"] == k0["r_p"]
        assert kb["r_d"] == k0["r_d"]
        assert dual_violation(P._Modified(lp, zero_bounds=True), y) == dual_violation(lp, y)


def test_phases_reach_feasibility_by_direct_evaluation():
    lp = polish_lp()
    eps = 1e-8
    # from the solve's state after 3,000 iterations (the polished solve's
    # successful attempt comes at the check t = 3,072)
    mid = mid_point(lp, 3000)
    got = P.feasibility_polish(lp, P.Opts(eps_rel=eps, eps_gap=1e-4), mid.x, mid.y, mid.eta,
                               mid.omega, 3000)
    assert got["kkt"] is not None
    nb = P.bhat_norm(np.asarray(lp.row_lo, float), np.asarray(lp.row_hi, float))
    rp, cv = primal_violation(lp, got["x"])
    # (the column bounds hold up to the rounding of the unscaling)
    assert rp <= eps * (1.0 + nb) and cv <= 1e-14 * (1.0 + np.max(np.abs(got["x"])))
    assert dual_violation(lp, got["y"]) <= eps * (1.0 + np.linalg.norm(lp.c))
    # both phases stayed near their start
    assert np.linalg.norm(got["x"] - mid.x) <= 0.1 * np.linalg.norm(mid.x)
    assert np.linalg.norm(got["y"] - mid.y) <= 0.1 * np.linalg.norm(mid.y)


def test_polished_solve_meets_the_test_and_the_optimum():
    lp = polish_lp()
    p_star, _, _ = highs_solve(lp)
    plain = P.pdhg_solve(lp, P.Opts(eps_rel=1e-8, eps_gap=1e-4))
    r = P.pdhg_solve(lp, P.Opts(eps_rel=1e-8, eps_gap=1e-4, polish=True))
    assert r.status == P.OPTIMAL and r.polish["successes"] == 1
    assert r.iterations < plain.iterations
    nb = P.bhat_norm(np.asarray(lp.row_lo, float), np.asarray(lp.row_hi, float))
    rp, cv = primal_violation(lp, r.x)
    assert rp <= 1e-8 * (1.0 + nb) and cv <= 1e-14 * (1.0 + np.max(np.abs(r.x)))
    assert dual_violation(lp, r.y) <= 1e-8 * (1.0 + np.linalg.norm(lp.c))
    # a relative gap of 1e-4 bounds the objective error by about that much
    assert abs(r.kkt["p"] - p_star) <= 2e-4 * (1.0 + abs(p_star))


def test_separate_gap_tolerance_defaults_to_eps_rel():
    lp = lpgen.c1_small()
    a = P.pdhg_solve(lp, P.Opts())
    b = P.pdhg_solve(lp, P.Opts(eps_gap=1e-6))
    assert a.iterations == b.iterations and np.array_equal(a.x, b.x)
    # a looser gap tolerance never stops later
    c = P.pdhg_solve(lp, P.Opts(eps_gap=1e-3))
    assert c.iterations <= a.iterations
    assert P.kkt_met(c.kkt, P.Opts(eps_gap=1e-3))


def test_failed_attempts_leave_the_main_trajectory_alone():
    # on this LP every attempt fails at eps_gap = eps_rel (the pair's gap
    # grows): the main iterates equal the plain solve's, and the phases only
    # add iterations
    lp = lpgen.general_structure(2000, 5000, 6, nnz_target=40_000, one_sided=0.2)
    plain = P.pdhg_solve(lp, P.Opts())
    r = P.pdhg_solve(lp, P.Opts(polish=True))
    assert r.polish["attempts"] >= 1 and r.polish["successes"] == 0
    assert np.array_equal(r.x_iter, plain.x_iter) and np.array_equal(r.y_iter, plain.y_iter)
    assert r.iterations == plain.iterations + r.polish["phase_iterations"]
    assert r.restarts == plain.restarts


def test_polish_budget_rounds_up_to_a_check_period():
    # max(K, fraction t) rounded up to a multiple of K, at least one period
    lp = lpgen.c1_small()
    mid = mid_point(lp, 200)
    opts = P.Opts(eps_rel=1e-12, eps_gap=1e-4, polish_fraction=0.01)
    got = P.feasibility_polish(lp, opts, mid.x, mid.y, mid.eta, mid.omega, 200)
    # eps 1e-12 is out of reach: the primal phase uses its whole budget, K
    assert got["kkt"] is None and got["iterations"] == 64
