"""Pins for the oracle presolve/postsolve (CPU only).

The worked examples of Sec. 2 (fix a variable, the redundant row
x1 >= 1, x2 >= 2, x1 + 2 x2 >= 5, the doubleton x1 + x2 = 1 with x >= 0) and
the invariant that postsolve(exact solution of presolve(LP)) is a KKT point of
the original LP with the planted optimal objective.  Exact reduced solutions
come from scipy's HiGHS, independent of the oracle's PDHG.
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import presolve as PS
from lp_helpers import SimpleLP, highs_solve

INF = np.inf


def solve_via_presolve(lp):
    res = PS.presolve(lp)
    assert res.status in (PS.REDUCED, PS.SOLVED)
    red = res.reduced
    if red.m == 0 and red.n == 0:
        xr, yr = np.zeros(0), np.zeros(0)
    elif red.m == 0:
        # no rows left: each column at the bound its cost points to
        xr = np.where(red.c > 0, red.col_lo, np.where(red.c < 0, red.col_hi,
                                                      np.clip(0.0, red.col_lo, red.col_hi)))
        yr = np.zeros(0)
    else:
        _, xr, yr = highs_solve(red)
    x, y, z = PS.postsolve(res, xr, yr)
    return res, x, y, z


def test_fix_variable_postsolve_sets_reduced_cost():
    # Sec. 2.1: x_k fixed at xhat; postsolve x_k = xhat, y unchanged,
    # z_k = c_k - a_k^T y
    A = [[1.0, 2.0, 1.0], [3.0, 1.0, -1.0]]
    lp = SimpleLP(A, [1.0, 2.0, -1.0], [2.0, 1.0], [INF, INF], [0.0, 0.5, 0.0],
                  [10.0, 0.5, 10.0])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["fixed_col"] == 1
    assert x[1] == 0.5
    assert abs(z[1] - (2.0 - (2.0 * y[0] + 1.0 * y[1]))) <= 1e-12
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9
    p, _, _ = highs_solve(lp)
    assert abs(k["p"] - p) <= 1e-9 * (1 + abs(p))


def test_redundant_row_worked_example():
    # x1 >= 1, x2 >= 2 imply x1 + 2 x2 >= 5: the row is removed
    lp = SimpleLP([[1.0, 2.0]], [1.0, 1.0], [5.0], [INF], [1.0, 2.0], [INF, INF])
    res = PS.presolve(lp)
    assert res.counts["redundant_row"] == 1
    assert res.reduced.m == 0
    _, x, y, _ = solve_via_presolve(lp)
    assert y[0] == 0.0 and list(x) == [1.0, 2.0]


def test_doubleton_worked_example():
    # x1 + x2 = 1, x >= 0: x1's bound x1 >= 0 moves to x2 <= 1, x1 = 1 - x2,
    # row and x1 removed; a reduced x2 = a maps back to (1 - a, a)
    lp = SimpleLP([[1.0, 1.0]], [2.0, 3.0], [1.0], [1.0], [0.0, 0.0], [INF, INF])
    ps = PS.Presolver(lp)
    ps.doubleton(0)
    assert ps.records[0][0] == "doubleton" and ps.records[0][2] == 0  # x1 eliminated
    assert ps.lx[1] == 0.0 and ps.ux[1] == 1.0
    assert not ps.row_on[0] and not ps.col_on[0]
    red, rmap, cmap = ps.reduced()
    res = PS.PresolveResult(PS.REDUCED, red, rmap, cmap, ps.records, 1, m0=1, n0=2)
    for a in (0.0, 0.25, 1.0):
        x, _, _ = PS.postsolve(res, np.array([a]), np.zeros(0))
        assert x[0] == 1.0 - a and x[1] == a
    # objective 2 x1 + 3 x2 = 2 + x2 -> min at x2 = 0, x = (1, 0), p = 2
    _, x, y, z = solve_via_presolve(lp)
    assert np.allclose(x, [1.0, 0.0])
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-12 and abs(k["p"] - 2.0) <= 1e-12


@pytest.mark.parametrize("a,lo,hi,c", [
    (2.0, 1.0, 3.0, 1.0), (2.0, 1.0, 3.0, -1.0), (-2.0, 1.0, 3.0, 1.0),
    (-2.0, 1.0, 3.0, -1.0), (0.5, -INF, 1.0, -1.0), (-0.5, -1.0, INF, -1.0),
])
def test_singleton_row_duals_both_signs(a, lo, hi, c):
    # one singleton row tightening a boxed variable, plus a second row so the
    # LP is not trivial
    A = [[a, 0.0], [1.0, 1.0]]
    lp = SimpleLP(A, [c, 0.5], [lo, 0.0], [hi, 4.0], [-5.0, 0.0], [5.0, 3.0])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["singleton_row"] >= 1
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9
    p, _, _ = highs_solve(lp)
    assert abs(k["p"] - p) <= 1e-9 * (1 + abs(p))


@pytest.mark.parametrize("c0,c1", [(2.0, 3.0), (3.0, 2.0), (-1.0, 1.0), (1.0, -4.0)])
def test_doubleton_postsolve_both_branches(c0, c1):
    # x0 + 2 x1 = 2 with boxes; a third column linking another row so the
    # eliminated column has an entry elsewhere (substitution + fill-in)
    A = [[1.0, 2.0, 0.0], [1.0, 0.0, 1.0]]
    lp = SimpleLP(A, [c0, c1, 0.3], [2.0, 0.5], [2.0, 3.0], [0.0, 0.0, -1.0],
                  [1.5, 5.0, 2.0])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["doubleton"] >= 1
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9
    p, _, _ = highs_solve(lp)
    assert abs(k["p"] - p) <= 1e-9 * (1 + abs(p))


def test_free_column_singleton():
    # x2 is free and appears only in the equality row 0
    A = [[1.0, 1.0, 2.0], [1.0, -1.0, 0.0]]
    lp = SimpleLP(A, [1.0, 2.0, -1.0], [4.0, -1.0], [4.0, 3.0], [0.0, 0.0, -INF],
                  [5.0, 5.0, INF])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["free_col_singleton"] == 1
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9
    p, _, _ = highs_solve(lp)
    assert abs(k["p"] - p) <= 1e-9 * (1 + abs(p))


def test_infeasible_and_unbounded_detection():
    lp = SimpleLP(np.zeros((1, 1)), [1.0], [1.0], [2.0], [0.0], [1.0])  # empty row 1 <= 0
    assert PS.presolve(lp).status == PS.INFEASIBLE
    lp = SimpleLP([[1.0, 0.0], [1.0, 0.0]], [1.0, 0.0], [3.0, -INF], [INF, 1.0],
                  [0.0, 0.0], [INF, 1.0])  # x0 >= 3 and x0 <= 1
    assert PS.presolve(lp).status == PS.INFEASIBLE
    lp = SimpleLP([[1.0, 0.0]], [1.0, -1.0], [1.0], [2.0], [0.0, 0.0], [INF, INF])
    assert PS.presolve(lp).status == PS.UNBOUNDED  # empty col with c < 0, u = inf


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_postsolve_of_exact_reduced_solution_is_kkt(seed):
    lp = lpgen.general_structure(600, 1500, seed, nnz_target=9000, one_sided=0.2)
    res, x, y, z = solve_via_presolve(lp)
    red = res.reduced
    assert red.m < lp.m and red.n < lp.n
    assert sum(res.counts.values()) > 0
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))
    # dual feasibility is exact by construction of every postsolve step
    g = lp.c - lp.csr().T @ y
    assert np.max(np.abs(g - z)) <= 1e-8 * (1 + np.max(np.abs(lp.c)))


def test_presolve_scaled_c2_structure():
    lp = lpgen.c2_presolvable(scale=0.005)
    res, x, y, z = solve_via_presolve(lp)
    for key in ("empty_row", "fixed_col", "singleton_row", "doubleton"):
        assert res.counts[key] > 0, key
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8
    assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))


def test_pdhg_on_reduced_then_postsolve():
    lp = lpgen.general_structure(500, 1200, 41, nnz_target=7000)
    res = PS.presolve(lp)
    r = oracle.pdhg_solve(res.reduced, oracle.Opts(eps_rel=1e-8))
    assert r.status == 0
    x, y, z = PS.postsolve(res, r.x, r.y, r.z)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-6
    assert abs(k["p"] - lp.p_star) <= 1e-6 * (1 + abs(lp.p_star))


def test_variable_lock_worked_example():
    # Sec. 2.3: c_1 < 0 and no row keeps x_1 from increasing (x1 + x2 >= 1 has
    # no upper bound): every optimum has x_1 = 3, its upper bound
    lp = SimpleLP([[1.0, 1.0]], [-1.0, 1.0], [1.0], [INF], [0.0, 0.0], [3.0, INF])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["dual_fix"] == 1
    assert x[0] == 3.0 and x[1] == 0.0
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-12
    p, _, _ = highs_solve(lp)
    assert abs(k["p"] - p) <= 1e-12 * (1 + abs(p))
    assert z[0] < 0  # at its upper bound
    # the mirrored case: c > 0, the row only bounds x from above
    lp = SimpleLP([[1.0, -1.0]], [1.0, -1.0], [-INF], [2.0], [-1.0, 0.0], [4.0, 5.0])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["dual_fix"] >= 1
    k = oracle.rel_kkt(lp, x, y)
    p, _, _ = highs_solve(lp)
    assert k["rel_kkt"] <= 1e-12 and abs(k["p"] - p) <= 1e-12 * (1 + abs(p))


def test_variable_lock_unbounded():
    # c_1 < 0, no up-lock, no upper bound: the (feasible) LP is unbounded
    lp = SimpleLP([[1.0, 1.0]], [-1.0, 1.0], [1.0], [INF], [0.0, 0.0], [INF, INF])
    assert PS.presolve(lp).status == PS.UNBOUNDED


def test_variable_locks_on_one_sided_rows_keep_the_optimum():
    # rows A x >= b with A >= 0: every column with c_j < 0 and a finite upper
    # bound has no up-lock and is fixed there; the optimum is unchanged
    rng = np.random.default_rng(11)
    m, n = 40, 90
    A = (rng.random((m, n)) < 0.12) * rng.uniform(0.5, 2.0, (m, n))
    A[np.arange(m), rng.integers(0, n, m)] += 1.0  # no empty rows
    c = rng.normal(size=n)
    lp = SimpleLP(A, c, rng.uniform(0.5, 1.5, m), np.full(m, INF), np.zeros(n),
                  rng.uniform(1.0, 3.0, n))
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["dual_fix"] >= int(np.sum(c < 0)) // 2
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8
    p, _, _ = highs_solve(lp)
    assert abs(k["p"] - p) <= 1e-8 * (1 + abs(p))


def test_variable_lock_respects_the_coefficient_sign():
    # -x1 + x2 >= 1: increasing x1 would violate the row (a < 0 with a finite
    # lower side is an up-lock), so c_1 < 0 does not fix x1; the optimum is
    # x = (0, 1) with objective 2, while fixing x1 at 4 would give 6
    lp = SimpleLP([[-1.0, 1.0]], [-1.0, 2.0], [1.0], [INF], [0.0, 0.0], [4.0, 10.0])
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["dual_fix"] == 0
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-12 and abs(k["p"] - 2.0) <= 1e-12


# Column singleton x0 in the ranged row 1 <= a x0 + x1 + x2 <= 6, with
# x1 - x2 in [-2, 2] and 0 <= x1, x2 <= 10; (a, c0, l0, u0, side) where side
# is the row side every optimum sits at (+1 lower, -1 upper).
_INEQ_CASES = [
    (-1.0, -1.0, 0.0, INF, 1),    # only l finite, a < 0, c < 0: y >= q > 0
    (1.0, -1.0, 0.0, INF, -1),    # only l finite, a > 0, c < 0: y <= q < 0
    (2.0, 1.0, -INF, 5.0, 1),     # only u finite, a > 0, c > 0: y >= q > 0
    (-2.0, 1.0, -INF, 5.0, -1),   # only u finite, a < 0, c > 0: y <= q < 0
    (1.0, 2.0, -INF, INF, 1),     # free: y = q > 0
    (1.0, -0.5, -INF, INF, -1),   # free: y = q < 0
]


def _ineq_lp(a, c0, l0, u0):
    return SimpleLP([[a, 1.0, 1.0], [0.0, 1.0, -1.0]], [c0, 1.0, 0.5], [1.0, -2.0], [6.0, 2.0],
                    [l0, 0.0, 0.0], [u0, 10.0, 10.0])


@pytest.mark.parametrize("a,c0,l0,u0,side", _INEQ_CASES)
def test_column_singleton_in_inequality_picks_the_active_side(a, c0, l0, u0, side):
    lp = _ineq_lp(a, c0, l0, u0)
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["ineq_to_eq"] == 1
    # every optimum has row 0 at that side: HiGHS's optimum on the original
    # LP does, and its dual has the matching strict sign
    p, xh, yh = highs_solve(lp)
    act = a * xh[0] + xh[1] + xh[2]
    assert abs(act - (1.0 if side > 0 else 6.0)) <= 1e-9
    assert yh[0] * side > 0
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9
    assert abs(k["p"] - p) <= 1e-9 * (1 + abs(p))
    assert y[0] * side > 0


def test_column_singleton_in_inequality_not_applied_without_a_sign():
    # boxed x0, or a cost that does not push y away from 0: no conversion
    for a, c0, l0, u0 in [(1.0, -1.0, 0.0, 3.0), (-1.0, 1.0, 0.0, INF), (1.0, 0.0, -INF, INF)]:
        res = PS.presolve(_ineq_lp(a, c0, l0, u0))
        assert res.counts["ineq_to_eq"] == 0


def test_column_singleton_in_inequality_postsolve_clamps_a_wrong_signed_dual():
    lp = _ineq_lp(-1.0, -1.0, 0.0, INF)
    res = PS.presolve(lp)
    assert res.counts["ineq_to_eq"] == 1 and 0 in list(res.row_map)
    red = res.reduced
    rng = np.random.default_rng(3)
    xr = rng.uniform(0.0, 1.0, red.n)
    yr = rng.normal(size=red.m)
    yr[list(res.row_map).index(0)] = -0.25  # wrong sign for a lower side
    x, y, z = PS.postsolve(res, xr, yr)
    assert y[0] == 0.0
    # dual feasibility c - A^T y - z = 0 survives the clamp
    g = lp.c - lp.csr().T @ y
    assert np.max(np.abs(g - z)) <= 1e-12


def test_parallel_rows_worked_example():
    # x0 + 2 x1 >= 1 and 2 x0 + 4 x1 <= 10 are one row 1 <= x0 + 2 x1 <= 5;
    # -3 x0 - 6 x1 >= -12 tightens it to <= 4
    A = [[1.0, 2.0, 0.0], [2.0, 4.0, 0.0], [-3.0, -6.0, 0.0], [1.0, 0.0, 1.0]]
    lp = SimpleLP(A, [-1.0, -1.0, 1.0], [1.0, -INF, -12.0, 0.5], [INF, 10.0, INF, INF],
                  [0.0, 0.0, 0.0], [INF, INF, INF])
    res = PS.presolve(lp)
    assert res.counts["parallel_row"] == 2
    par = [r for r in res.records if r[0] == "parallel_row"]
    # (kept row, merged row, s, lower side from the merged row, upper side from it)
    assert par == [("parallel_row", 0, 1, 2.0, False, True),
                   ("parallel_row", 0, 2, -3.0, False, True)]
    _, x, y, z = solve_via_presolve(lp)
    p, _, _ = highs_solve(lp)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9 and abs(k["p"] - p) <= 1e-9 * (1 + abs(p))
    # the active side x0 + 2 x1 <= 4 came from row 2 (s = -3): its dual is
    # y_0 / s >= 0 there, rows 0 and 1 carry none
    assert y[1] == 0.0 and y[0] == 0.0 and y[2] > 0


def test_parallel_rows_infeasible():
    lp = SimpleLP([[1.0, 1.0], [2.0, 2.0]], [1.0, 1.0], [5.0, -INF], [INF, 4.0],
                  [0.0, 0.0], [INF, INF])
    assert PS.presolve(lp).status == PS.INFEASIBLE


@pytest.mark.parametrize("seed", [5, 6])
def test_parallel_rows_planted_copies(seed):
    # copies of random rows scaled by s (either sign), some with bounds that
    # cut the optimum, and near-parallel copies (1e-6 off) that must stay
    base = lpgen.general_structure(120, 300, seed, nnz_target=1500, one_sided=0.3)
    A = base.csr().toarray()
    lo, hi = base.row_lo.copy(), base.row_hi.copy()
    rng = np.random.default_rng(seed)
    rows = rng.choice(base.m, 30, replace=False)
    extra_A, extra_lo, extra_hi = [], [], []
    for t, i in enumerate(rows):
        s = rng.choice([-3.0, -0.5, 0.25, 2.0, 7.0])
        a = s * A[i]
        act = A[i] @ base.x_star
        l, h = act - rng.uniform(0.0, 2.0), act + rng.uniform(0.0, 2.0)
        if t % 3 == 2:
            a = a * (1.0 + 1e-6 * (np.arange(base.n) % 2))
        if s > 0:
            extra_lo.append(s * l)
            extra_hi.append(s * h if t % 2 else INF)
        else:
            extra_lo.append(s * h if t % 2 else -INF)
            extra_hi.append(s * l)
        extra_A.append(a)
    lp = SimpleLP(np.vstack([A, extra_A]), base.c, np.concatenate([lo, extra_lo]),
                  np.concatenate([hi, extra_hi]), base.col_lo, base.col_hi)
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["parallel_row"] >= 15
    p, _, _ = highs_solve(lp)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8
    assert abs(k["p"] - p) <= 1e-8 * (1 + abs(p))
    g = lp.c - lp.csr().T @ y
    assert np.max(np.abs(g - z)) <= 1e-8 * (1 + np.max(np.abs(lp.c)))


@pytest.mark.parametrize("seed", [13, 14])
def test_medium_structure_keeps_the_planted_optimum(seed):
    # planted parallel copies and slack column singletons: both explorers
    # fire, and postsolve of the exact reduced solution is optimal
    lp = lpgen.medium_structure(600, 1500, seed, nnz_target=9000)
    res, x, y, z = solve_via_presolve(lp)
    assert res.counts["parallel_row"] >= lp.meta["parallel"] // 2
    assert res.counts["ineq_to_eq"] >= lp.meta["slack"] // 2
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8
    assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))


def test_rounding_residue_in_a_cost_is_not_a_sign():
    # a cost of -1e-16 (what substitutions leave of a structurally zero cost)
    # must neither fix x0 at its infinite upper bound ("unbounded") nor make
    # row 0 an equality; the LP is bounded with optimum 1 at x = (0, 1) or any
    # point with x0 + x1 >= 1, x1 >= 1
    lp = SimpleLP([[1.0, 1.0], [0.0, 1.0]], [-1e-16, 1.0], [1.0, 1.0], [INF, INF],
                  [0.0, 0.0], [INF, INF])
    res, x, y, z = solve_via_presolve(lp)
    assert res.status in (PS.REDUCED, PS.SOLVED)
    assert res.counts["dual_fix"] == 0 and res.counts["ineq_to_eq"] == 0
    assert abs(float(lp.c @ x) - 1.0) <= 1e-12
    # an empty column with such a cost sits at proj(0), not at an infinite bound
    lp = SimpleLP([[0.0, 1.0]], [-1e-17, 1.0], [1.0], [INF], [0.0, 0.0], [INF, INF])
    res, x, y, z = solve_via_presolve(lp)
    assert res.status == PS.SOLVED and res.counts["empty_col"] == 2
    assert x[0] == 0.0 and x[1] == 1.0


def test_medium_instance_that_met_cost_residue_stays_bounded():
    # the instance on which a -1.1e-16 cost left by free-column-singleton
    # substitutions was once taken for a sign; its planted optimum is finite
    import suite

    lp = suite.make_instance(300000, 2010)
    res = PS.presolve(lp)
    assert res.status == PS.REDUCED


# ---------------------------------------------------------------------------
# primal propagation (opt-in medium explorer)

def solve_via_presolve_prop(lp):
    res = PS.presolve(lp, propagation=True)
    assert res.status in (PS.REDUCED, PS.SOLVED)
    red = res.reduced
    if red.m == 0:
        xr = np.where(red.c > 0, red.col_lo, np.where(red.c < 0, red.col_hi,
                                                      np.clip(0.0, red.col_lo, red.col_hi)))
        yr = np.zeros(0)
    else:
        _, xr, yr = highs_solve(red)
    x, y, z = PS.postsolve(res, xr, yr)
    return res, x, y, z


def test_propagation_worked_example():
    # x1 + x2 >= 3 with x2 <= 1 implies x1 >= 2; min x1 + 0.5 x2 puts x2 at 1
    # and x1 at the implied bound, whose reduced cost moves to the row
    lp = SimpleLP([[1.0, 1.0], [1.0, -1.0]], [1.0, 0.5], [3.0, -20.0], [np.inf, 20.0],
                  [0.0, 0.0], [10.0, 1.0])
    res, x, y, z = solve_via_presolve_prop(lp)
    tight = [r for r in res.records if r[0] == "tighten"]
    assert any(r[1] == 0 and r[2] == 0 and r[4] == 0 for r in tight)  # x1's lower from row 0
    assert abs(res.reduced.col_lo[list(res.col_map).index(0)] - 2.0) <= 1e-15
    p, _, _ = highs_solve(lp)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9 and abs(k["p"] - p) <= 1e-9 * (1 + abs(p))
    assert abs(x[0] - 2.0) <= 1e-9 and y[0] > 0 and abs(z[0]) <= 1e-12


def test_propagation_proves_infeasibility():
    # x1 + x2 >= 3 with both at most 1
    lp = SimpleLP([[1.0, 1.0], [1.0, -1.0]], [1.0, 1.0], [3.0, -5.0], [np.inf, 5.0],
                  [0.0, 0.0], [1.0, 1.0])
    assert PS.presolve(lp).status == PS.REDUCED  # the fast rules alone do not see it
    assert PS.presolve(lp, propagation=True).status == PS.INFEASIBLE


@pytest.mark.parametrize("make", [
    lambda: lpgen.general_structure(600, 1500, 31, nnz_target=9000, one_sided=0.2),
    lambda: lpgen.medium_structure(600, 1500, 13, nnz_target=9000),
    lambda: lpgen.c2_presolvable(scale=0.005),
])
def test_propagation_keeps_the_planted_optimum(make):
    lp = make()
    res, x, y, z = solve_via_presolve_prop(lp)
    assert res.counts["tightened"] > 0
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))
    g = lp.c - lp.csr().T @ y
    assert np.max(np.abs(g - z)) <= 1e-8 * (1 + np.max(np.abs(lp.c)))


# ---------------------------------------------------------------------------
# parallel columns (opt-in medium explorer)

def test_parallel_columns_worked_example():
    # column 2 is 2 x column 1 in every row and in the cost: x1 + 2 x2 acts as
    # one variable x' in [0, 1] + 2 [0, 2] = [0, 5], capped at 4 by row 0
    A = [[1.0, 2.0, 0.0], [1.0, 2.0, 1.0]]
    lp = SimpleLP(A, [-1.0, -2.0, 1.0], [-np.inf, 4.0], [4.0, np.inf], [0.0, 0.0, 0.0],
                  [1.0, 2.0, 10.0])
    res = PS.presolve(lp, parallel_cols=True)
    assert res.counts["parallel_col"] == 1
    rec = [r for r in res.records if r[0] == "parallel_col"][0]
    assert rec[1:4] == (0, 1, 2.0)
    red = res.reduced
    _, xr, yr = highs_solve(red) if red.m else (None, np.zeros(red.n), np.zeros(0))
    if red.m == 0:
        xr = np.where(red.c > 0, red.col_lo, np.where(red.c < 0, red.col_hi, 0.0))
    x, y, z = PS.postsolve(res, xr, yr)
    p, _, _ = highs_solve(lp)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9 and abs(k["p"] - p) <= 1e-9 * (1 + abs(p))
    assert 0.0 <= x[0] <= 1.0 and 0.0 <= x[1] <= 2.0


@pytest.mark.parametrize("seed", [13, 21])
def test_parallel_columns_keep_the_planted_optimum(seed):
    lp = lpgen.medium_structure(600, 1500, seed, nnz_target=9000, frac_parallel_cols=0.05)
    res = PS.presolve(lp, parallel_cols=True)
    assert res.counts["parallel_col"] >= 30
    red = res.reduced
    _, xr, yr = highs_solve(red)
    x, y, z = PS.postsolve(res, xr, yr)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))
    g = lp.c - lp.csr().T @ y
    assert np.max(np.abs(g - z)) <= 1e-8 * (1 + np.max(np.abs(lp.c)))
    assert np.all(x >= lp.col_lo - 1e-9) and np.all(x <= lp.col_hi + 1e-9)


def test_parallel_columns_need_parallel_costs():
    # same columns but c_2 != 2 c_1: not merged
    lp = SimpleLP([[1.0, 2.0], [1.0, 2.0]], [1.0, 3.0], [1.0, -5.0], [5.0, 5.0], [0.0, 0.0],
                  [4.0, 4.0])
    assert PS.presolve(lp, parallel_cols=True).counts["parallel_col"] == 0


# ---------------------------------------------------------------------------
# dual propagation (opt-in medium explorer)

def _dual_prop_example():
    # x1 >= 0 with c1 = -3 in x1 + x2 >= 1 (y0 >= 0) and x1 - x3 <= 5 (y1 <= 0):
    # its dual constraint y0 + y1 <= -3 forces y1 <= -3, so row 1 is active at
    # its upper side in every optimum (variable locks and column singletons
    # see nothing here)
    return SimpleLP([[1.0, 1.0, 0.0], [1.0, 0.0, -1.0]], [-3.0, 1.0, 0.0], [1.0, -np.inf],
                    [np.inf, 5.0], [0.0, 0.0, 0.0], [np.inf, np.inf, 10.0])


def test_dual_propagation_worked_example():
    lp = _dual_prop_example()
    assert PS.presolve(lp).counts["ineq_to_eq"] == 0
    res = PS.presolve(lp, dual_propagation=True)
    assert res.counts["dual_prop"] >= 1
    assert ("row_to_eq", 1, -1) == [r for r in res.records if r[0] == "row_to_eq"][0][:3]
    p, xh, yh = highs_solve(lp)
    assert abs(xh[0] - xh[2] - 5.0) <= 1e-9 and yh[1] <= -3.0 + 1e-9
    red = res.reduced
    if red.m:
        _, xr, yr = highs_solve(red)
    else:
        xr = np.where(red.c > 0, red.col_lo, np.where(red.c < 0, red.col_hi, 0.0))
        yr = np.zeros(0)
    x, y, z = PS.postsolve(res, xr, yr)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-9 and abs(k["p"] - p) <= 1e-9 * (1 + abs(p))


@pytest.mark.parametrize("make", [
    lambda: lpgen.general_structure(600, 1500, 31, nnz_target=9000, one_sided=0.2),
    lambda: lpgen.medium_structure(600, 1500, 13, nnz_target=9000),
    lambda: lpgen.c2_presolvable(scale=0.005),
])
def test_dual_propagation_keeps_the_planted_optimum(make):
    lp = make()
    res = PS.presolve(lp, dual_propagation=True)
    _, xr, yr = highs_solve(res.reduced)
    x, y, z = PS.postsolve(res, xr, yr)
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-8, k
    assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))
