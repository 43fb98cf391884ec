"""Host C presolve/postsolve (through the C ABI) against the oracle (CPU only).

Presolve is integer and index work plus deterministic IEEE arithmetic, so the
reduced problems must agree exactly: same sizes, same kept rows and columns,
same sparsity pattern, and bit-identical values.  Postsolve outputs agree to
1e-12 relative (same formulas, summation order may differ).
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import presolve as PS
from lp_helpers import SimpleLP, highs_solve

pkg = pytest.importorskip("paper_2604_23951_gb300")

INF = np.inf


def _lib_or_skip():
    try:
        pkg.load()
    except RuntimeError as e:  # library not built in this checkout
        pytest.skip(str(e))


def _one_sided_rows(seed=11, m=40, n=90):
    # A x >= b with A >= 0: the variable-lock explorer fixes many columns
    rng = np.random.default_rng(seed)
    A = (rng.random((m, n)) < 0.12) * rng.uniform(0.5, 2.0, (m, n))
    A[np.arange(m), rng.integers(0, n, m)] += 1.0
    return SimpleLP(A, rng.normal(size=n), rng.uniform(0.5, 1.5, m), np.full(m, INF),
                    np.zeros(n), rng.uniform(1.0, 3.0, n))


def _parallel_example():
    A = [[1.0, 2.0, 0.0], [2.0, 4.0, 0.0], [-3.0, -6.0, 0.0], [1.0, 0.0, 1.0]]
    return SimpleLP(A, [-1.0, -1.0, 1.0], [1.0, -INF, -12.0, 0.5], [INF, 10.0, INF, INF],
                    [0.0, 0.0, 0.0], [INF, INF, INF])


def _ineq_singletons():
    # column singletons in inequality rows with every sign combination, one
    # block of two rows and three columns each
    blocks = [(-1.0, -1.0, 0.0, INF), (1.0, -1.0, 0.0, INF), (2.0, 1.0, -INF, 5.0),
              (-2.0, 1.0, -INF, 5.0), (1.0, 2.0, -INF, INF), (1.0, -0.5, -INF, INF)]
    k = len(blocks)
    A = np.zeros((2 * k, 3 * k))
    c = np.zeros(3 * k)
    lo, hi = np.zeros(2 * k), np.zeros(2 * k)
    lx, ux = np.zeros(3 * k), np.zeros(3 * k)
    for t, (a, c0, l0, u0) in enumerate(blocks):
        A[2 * t, 3 * t:3 * t + 3] = [a, 1.0, 1.0]
        A[2 * t + 1, 3 * t + 1:3 * t + 3] = [1.0, -1.0]
        c[3 * t:3 * t + 3] = [c0, 1.0, 0.5]
        lo[2 * t:2 * t + 2] = [1.0, -2.0]
        hi[2 * t:2 * t + 2] = [6.0, 2.0]
        lx[3 * t:3 * t + 3] = [l0, 0.0, 0.0]
        ux[3 * t:3 * t + 3] = [u0, 10.0, 10.0]
    return SimpleLP(A, c, lo, hi, lx, ux)


def _cases():
    return [
        ("medium", lambda: lpgen.medium_structure(600, 1500, 13, nnz_target=9000)),
        ("variable_locks", _one_sided_rows),
        ("general_small", lambda: lpgen.general_structure(600, 1500, 31, nnz_target=9000,
                                                          one_sided=0.2)),
        ("general_b", lambda: lpgen.general_structure(800, 2000, 77, nnz_target=16000)),
        ("c2_scaled", lambda: lpgen.c2_presolvable(scale=0.01)),
        ("c1", lambda: lpgen.c1_small()),
        ("tiny_box", lambda: lpgen.tiny_box(5, 6, 9)),
        ("doubleton_chain", lambda: SimpleLP(
            [[1.0, 1.0, 0.0, 0.0], [0.0, 1.0, -2.0, 0.0], [0.0, 0.0, 1.0, 3.0],
             [1.0, 0.0, 1.0, 1.0]],
            [1.0, 2.0, -1.0, 0.5], [1.0, 0.0, 2.0, -INF], [1.0, 0.0, 2.0, 6.0],
            [0.0, 0.0, -1.0, 0.0], [INF, 5.0, 4.0, INF])),
        ("parallel_example", _parallel_example),
        ("ineq_singletons", _ineq_singletons),
        ("medium_b", lambda: lpgen.medium_structure(900, 2000, 29, nnz_target=15000,
                                                    frac_parallel=0.2, frac_slack=0.1)),
    ]


@pytest.mark.parametrize("name,make", _cases())
def test_reduced_problem_identical(name, make):
    _lib_or_skip()
    lp = make()
    ref = PS.presolve(lp)
    prob = pkg.Problem(lp, None)
    info = prob.presolve()
    assert info.status == ref.status
    red = prob.data()
    r = ref.reduced
    assert (red.m, red.n) == (r.m, r.n), name
    assert info.rounds == ref.rounds
    assert list(info.counts) == [ref.counts[k] for k in (
        "empty_row", "empty_col", "fixed_col", "singleton_row", "redundant_row",
        "dropped_side", "doubleton", "free_col_singleton", "dual_fix", "ineq_to_eq",
        "parallel_row", "tightened", "parallel_col", "dual_prop")] + [0, 0]
    np.testing.assert_array_equal(red.row_ptr, r.row_ptr)
    np.testing.assert_array_equal(red.col_idx, r.col_idx)
    np.testing.assert_array_equal(red.val, r.val)
    np.testing.assert_array_equal(red.c, r.c)
    np.testing.assert_array_equal(red.row_lo, r.row_lo)
    np.testing.assert_array_equal(red.row_hi, r.row_hi)
    np.testing.assert_array_equal(red.col_lo, r.col_lo)
    np.testing.assert_array_equal(red.col_hi, r.col_hi)
    assert red.obj_offset == r.obj_offset


@pytest.mark.parametrize("name,make", _cases()[:4])
def test_postsolve_matches_oracle_and_is_kkt(name, make):
    _lib_or_skip()
    lp = make()
    ref = PS.presolve(lp)
    prob = pkg.Problem(lp, None)
    prob.presolve()
    red = ref.reduced
    if red.m == 0:
        pytest.skip("nothing left to solve")
    _, xr, yr = highs_solve(red)
    xo, yo, zo = PS.postsolve(ref, xr, yr)
    xc, yc, zc = prob.postsolve_from(xr, yr)
    scale = 1 + max(np.max(np.abs(xo)), np.max(np.abs(yo)), np.max(np.abs(zo)))
    assert np.max(np.abs(xc - xo)) <= 1e-12 * scale
    assert np.max(np.abs(yc - yo)) <= 1e-12 * scale
    assert np.max(np.abs(zc - zo)) <= 1e-12 * scale
    k = oracle.rel_kkt(lp, xc, yc)
    assert k["rel_kkt"] <= 1e-8
    if np.isfinite(lp.p_star if hasattr(lp, "p_star") else np.nan):
        assert abs(k["p"] - lp.p_star) <= 1e-8 * (1 + abs(lp.p_star))


def test_host_rel_kkt_matches_oracle():
    _lib_or_skip()
    lp = lpgen.general_structure(300, 700, 5, nnz_target=4000, one_sided=0.3)
    prob = pkg.Problem(lp, None)
    rng = np.random.default_rng(0)
    x = lp.x_star + 0.01 * rng.standard_normal(lp.n)
    y = lp.y_star + 0.01 * rng.standard_normal(lp.m)
    a = prob.rel_kkt(x, y)
    b = oracle.rel_kkt(lp, x, y)
    for k in ("rel_kkt", "rel_p", "rel_d", "rel_gap", "p", "d"):
        assert abs(a[k] - b[k]) <= 1e-12 * (1 + abs(b[k])), k


@pytest.mark.parametrize("bad", ["nan_val", "bad_ptr", "dup_col", "lo_gt_hi", "col_range"])
def test_create_rejects_malformed_input(bad):
    _lib_or_skip()
    lp = lpgen.tiny_box(3, 4, 1)
    if bad == "nan_val":
        lp.val = lp.val.copy()
        lp.val[0] = np.nan
    elif bad == "bad_ptr":
        lp.row_ptr = lp.row_ptr.copy()
        lp.row_ptr[1], lp.row_ptr[2] = lp.row_ptr[2], lp.row_ptr[1]
    elif bad == "dup_col":
        lp.col_idx = lp.col_idx.copy()
        lp.col_idx[1] = lp.col_idx[0]
    elif bad == "lo_gt_hi":
        lp.col_lo = lp.col_lo.copy()
        lp.col_lo[0] = lp.col_hi[0] + 1
    elif bad == "col_range":
        lp.col_idx = lp.col_idx.copy()
        lp.col_idx[-1] = lp.n + 3
    with pytest.raises(pkg.LPError) as ei:
        pkg.Problem(lp, None)
    assert ei.value.code == -1


def test_solve_without_device_is_state_error():
    _lib_or_skip()
    prob = pkg.Problem(lpgen.tiny_box(3, 4, 1), None)
    with pytest.raises(pkg.LPError) as ei:
        prob.solve()
    assert ei.value.code == -4


@pytest.mark.parametrize("name,make", [c for c in _cases() if c[0] in
                                       ("medium", "medium_b", "ineq_singletons")])
def test_postsolve_matches_oracle_on_perturbed_solutions(name, make):
    # an approximate reduced solution (exact + noise) takes the branches an
    # exact one does not: wrong-signed duals of rows made equalities,
    # merged-row duals of either sign
    _lib_or_skip()
    lp = make()
    ref = PS.presolve(lp)
    prob = pkg.Problem(lp, None)
    prob.presolve()
    red = ref.reduced
    _, xr, yr = highs_solve(red)
    rng = np.random.default_rng(7)
    for scale in (1e-6, 1e-2, 1.0):
        xp = xr + scale * rng.standard_normal(red.n)
        yp = yr + scale * rng.standard_normal(red.m)
        xo, yo, zo = PS.postsolve(ref, xp, yp)
        xc, yc, zc = prob.postsolve_from(xp, yp)
        tol = 1e-12 * (1 + max(np.max(np.abs(xo)), np.max(np.abs(yo)), np.max(np.abs(zo))))
        assert np.max(np.abs(xc - xo)) <= tol
        assert np.max(np.abs(yc - yo)) <= tol
        assert np.max(np.abs(zc - zo)) <= tol
        # dual feasibility c - A^T y - z = 0 holds for any reduced solution
        g = lp.c - lp.csr().T @ yc
        assert np.max(np.abs(g - zc)) <= 1e-9 * (1 + np.max(np.abs(lp.c)))


def test_threaded_paths_match_oracle():
    # large enough for every threaded / batched path of the library: the
    # column store built by several threads (>= 1M nonzeros), the batched
    # fixed-column pass (>= 256 fixed columns, >= 4096 touched rows), the
    # parallel row hashing and reduced-problem build (>= 20000 rows)
    _lib_or_skip()
    lp = lpgen.medium_structure(42_000, 105_000, 17, nnz_target=1_000_000)
    assert lp.nnz >= 1_000_000
    ref = PS.presolve(lp)
    prob = pkg.Problem(lp, None)
    info = prob.presolve()
    assert info.status == ref.status and info.rounds == ref.rounds
    assert ref.counts["fixed_col"] >= 256
    red, r = prob.data(), ref.reduced
    assert (red.m, red.n) == (r.m, r.n)
    np.testing.assert_array_equal(red.row_ptr, r.row_ptr)
    np.testing.assert_array_equal(red.col_idx, r.col_idx)
    np.testing.assert_array_equal(red.val, r.val)
    np.testing.assert_array_equal(red.c, r.c)
    np.testing.assert_array_equal(red.row_lo, r.row_lo)
    np.testing.assert_array_equal(red.row_hi, r.row_hi)
    np.testing.assert_array_equal(red.col_lo, r.col_lo)
    np.testing.assert_array_equal(red.col_hi, r.col_hi)
    assert red.obj_offset == r.obj_offset


def _assert_same_reduced(prob, ref, info):
    assert info.status == ref.status and info.rounds == ref.rounds
    red, r = prob.data(), ref.reduced
    assert (red.m, red.n) == (r.m, r.n)
    np.testing.assert_array_equal(red.row_ptr, r.row_ptr)
    np.testing.assert_array_equal(red.col_idx, r.col_idx)
    np.testing.assert_array_equal(red.val, r.val)
    np.testing.assert_array_equal(red.c, r.c)
    np.testing.assert_array_equal(red.row_lo, r.row_lo)
    np.testing.assert_array_equal(red.row_hi, r.row_hi)
    np.testing.assert_array_equal(red.col_lo, r.col_lo)
    np.testing.assert_array_equal(red.col_hi, r.col_hi)
    assert red.obj_offset == r.obj_offset


@pytest.mark.parametrize("name,make", [c for c in _cases() if c[0] in
                                       ("medium", "general_small", "c2_scaled", "tiny_box",
                                        "medium_b", "variable_locks")])
def test_primal_propagation_matches_oracle(name, make):
    _lib_or_skip()
    lp = make()
    ref = PS.presolve(lp, propagation=True)
    prob = pkg.Problem(lp, None)
    info = prob.presolve(enable=pkg.LP_RULE_ALL | pkg.LP_RULE_PRIMAL_PROPAGATION)
    _assert_same_reduced(prob, ref, info)
    assert info.counts[11] == ref.counts["tightened"]
    if ref.reduced.m == 0 or ref.status != PS.REDUCED:
        return
    _, xr, yr = highs_solve(ref.reduced)
    rng = np.random.default_rng(1)
    for scale in (0.0, 1e-3):
        xp = xr + scale * rng.standard_normal(xr.shape[0])
        yp = yr + scale * rng.standard_normal(yr.shape[0])
        xo, yo, zo = PS.postsolve(ref, xp, yp)
        xc, yc, zc = prob.postsolve_from(xp, yp)
        tol = 1e-12 * (1 + max(np.max(np.abs(xo)), np.max(np.abs(yo)), np.max(np.abs(zo))))
        assert np.max(np.abs(xc - xo)) <= tol
        assert np.max(np.abs(yc - yo)) <= tol
        assert np.max(np.abs(zc - zo)) <= tol


def test_primal_propagation_infeasible_matches_oracle():
    _lib_or_skip()
    lp = SimpleLP([[1.0, 1.0], [1.0, -1.0]], [1.0, 1.0], [3.0, -5.0], [INF, 5.0],
                  [0.0, 0.0], [1.0, 1.0])
    prob = pkg.Problem(lp, None)
    info = prob.presolve(enable=pkg.LP_RULE_ALL | pkg.LP_RULE_PRIMAL_PROPAGATION)
    assert info.status == PS.INFEASIBLE == PS.presolve(lp, propagation=True).status


@pytest.mark.parametrize("seed", [13, 21])
def test_parallel_columns_match_oracle(seed):
    _lib_or_skip()
    lp = lpgen.medium_structure(600, 1500, seed, nnz_target=9000, frac_parallel_cols=0.05)
    ref = PS.presolve(lp, parallel_cols=True)
    prob = pkg.Problem(lp, None)
    info = prob.presolve(enable=pkg.LP_RULE_ALL | pkg.LP_RULE_PARALLEL_COLS)
    _assert_same_reduced(prob, ref, info)
    assert info.counts[12] == ref.counts["parallel_col"] > 0
    _, xr, yr = highs_solve(ref.reduced)
    rng = np.random.default_rng(2)
    for scale in (0.0, 1e-3):
        xp = xr + scale * rng.standard_normal(xr.shape[0])
        yp = yr + scale * rng.standard_normal(yr.shape[0])
        xo, yo, zo = PS.postsolve(ref, xp, yp)
        xc, yc, zc = prob.postsolve_from(xp, yp)
        tol = 1e-12 * (1 + max(np.max(np.abs(xo)), np.max(np.abs(yo)), np.max(np.abs(zo))))
        assert np.max(np.abs(xc - xo)) <= tol
        assert np.max(np.abs(yc - yo)) <= tol
        assert np.max(np.abs(zc - zo)) <= tol


def test_all_medium_explorers_together_match_oracle():
    _lib_or_skip()
    lp = lpgen.medium_structure(900, 2000, 29, nnz_target=15000, frac_parallel=0.2,
                                frac_slack=0.1, frac_parallel_cols=0.05)
    ref = PS.presolve(lp, propagation=True, parallel_cols=True, dual_propagation=True)
    prob = pkg.Problem(lp, None)
    info = prob.presolve(enable=pkg.LP_RULE_ALL | pkg.LP_RULE_PARALLEL_COLS
                         | pkg.LP_RULE_PRIMAL_PROPAGATION | pkg.LP_RULE_DUAL_PROPAGATION)
    _assert_same_reduced(prob, ref, info)


def _dual_prop_example():
    return SimpleLP([[1.0, 1.0, 0.0], [1.0, 0.0, -1.0]], [-3.0, 1.0, 0.0], [1.0, -INF],
                    [INF, 5.0], [0.0, 0.0, 0.0], [INF, INF, 10.0])


@pytest.mark.parametrize("name,make", [("example", _dual_prop_example)] +
                         [c for c in _cases() if c[0] in ("general_small", "medium", "c2_scaled",
                                                          "variable_locks", "ineq_singletons")])
def test_dual_propagation_matches_oracle(name, make):
    _lib_or_skip()
    lp = make()
    ref = PS.presolve(lp, dual_propagation=True)
    prob = pkg.Problem(lp, None)
    info = prob.presolve(enable=pkg.LP_RULE_ALL | pkg.LP_RULE_DUAL_PROPAGATION)
    _assert_same_reduced(prob, ref, info)
    assert info.counts[13] == ref.counts["dual_prop"]
    if ref.reduced.m == 0 or ref.status != PS.REDUCED:
        return
    _, xr, yr = highs_solve(ref.reduced)
    xo, yo, zo = PS.postsolve(ref, xr, yr)
    xc, yc, zc = prob.postsolve_from(xr, yr)
    tol = 1e-12 * (1 + max(np.max(np.abs(xo)), np.max(np.abs(yo)), np.max(np.abs(zo))))
    assert np.max(np.abs(xc - xo)) <= tol and np.max(np.abs(yc - yo)) <= tol
    assert np.max(np.abs(zc - zo)) <= tol
