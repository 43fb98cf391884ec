"""The paper's worked presolve examples (tests/golden/, each file citing its
section) against the oracle presolve and against the host C presolve through
the C ABI (CPU only).  The expected values are the ones the paper states; the
objective of an example, where the paper gives none, is the fixture's choice
and is said so in the file."""
import os

import numpy as np
import pytest

from oracle import presolve as PS
from lp_helpers import SimpleLP, highs_solve

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
COUNTS = ("empty_row", "empty_col", "fixed_col", "singleton_row", "redundant_row",
          "dropped_side", "doubleton", "free_col_singleton", "dual_fix", "ineq_to_eq",
          "parallel_row", "tightened", "parallel_col", "dual_prop")


def _word(w):
    try:
        return float(w)
    except ValueError:
        return w


def load(name):
    """key -> list of records (split on '|'), each a list of floats or words."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = line.split(":", 1)
            recs = []
            for part in val.split("|"):
                recs.append([_word(w) for w in part.split()])
            out[key.strip()] = recs
    return out


def lp_of(g, col_hi=None):
    return SimpleLP(g["A"], g["c"][0], g["row_lo"][0], g["row_hi"][0], g["col_lo"][0],
                    col_hi if col_hi is not None else g["col_hi"][0])


def capi():
    pkg = pytest.importorskip("paper_2604_23951_gb300")
    try:
        pkg.load()
    except RuntimeError as e:  # library not built in this checkout
        pytest.skip(str(e))
    return pkg


class Oracle:
    """Presolve, the reduced LP and postsolve through oracle/presolve.py."""

    def __init__(self, lp):
        self.res = PS.presolve(lp)
        self.status = self.res.status
        self.counts = dict(self.res.counts)
        self.reduced = self.res.reduced

    def postsolve(self, xr, yr):
        return PS.postsolve(self.res, xr, yr)


class Library:
    """The same through the C ABI (lp_presolve, lp_get_data, lp_postsolve_from)."""

    def __init__(self, lp, enable=None):
        pkg = capi()
        self.prob = pkg.Problem(lp, None)
        info = self.prob.presolve() if enable is None else self.prob.presolve(enable=enable)
        self.status = info.status
        self.counts = dict(zip(COUNTS, list(info.counts)))
        self.reduced = self.prob.data()

    def postsolve(self, xr, yr):
        return self.prob.postsolve_from(np.asarray(xr, float), np.asarray(yr, float))


def solve_reduced(side):
    red = side.reduced
    if red.m == 0:
        # no rows left: each column at the bound its cost points to
        c, lx, ux = (np.asarray(v, float) for v in (red.c, red.col_lo, red.col_hi))
        xr = np.where(c > 0, lx, np.where(c < 0, ux, np.clip(0.0, lx, ux)))
        return xr, np.zeros(0)
    _, xr, yr = highs_solve(red)
    return xr, yr


SIDES = [pytest.param(Oracle, id="oracle"), pytest.param(Library, id="library")]


@pytest.mark.parametrize("side", SIDES)
def test_fixing_a_variable(side):
    g = load("sec2_1_fixing_a_variable.txt")
    lp = lp_of(g)
    s = side(lp)
    rule, cnt = g["expect_count"][0]
    assert s.counts[rule] == cnt
    k, xhat = int(g["expect_fixed"][0][0]), g["expect_fixed"][0][1]
    x, y, z = s.postsolve(*solve_reduced(s))
    assert x[k] == xhat
    a_k = np.array([row[k] for row in g["A"]])
    assert abs(z[k] - (g["c"][0][k] - a_k @ y)) <= 1e-12
    p, _, _ = highs_solve(lp)
    assert abs(float(np.dot(g["c"][0], x)) - p) <= 1e-9 * (1 + abs(p))


@pytest.mark.parametrize("side", SIDES)
def test_redundant_constraint(side):
    g = load("sec2_2_redundant_constraint.txt")
    s = side(lp_of(g))
    rule, cnt = g["expect_count"][0]
    assert s.counts[rule] == cnt
    assert s.reduced.m == int(g["expect_reduced_rows"][0][0])
    x, y, _ = s.postsolve(*solve_reduced(s))
    assert list(x) == g["expect_x"][0] and list(y) == g["expect_y"][0]


def test_doubleton_row_oracle_pass():
    g = load("sec2_2_doubleton_row.txt")
    lp = lp_of(g)
    ps = PS.Presolver(lp)
    ps.doubleton(0)
    j = int(g["expect_doubleton_eliminates"][0][0])
    assert ps.records[0][0] == "doubleton" and ps.records[0][2] == j
    keep = 1 - j
    assert [ps.lx[keep], ps.ux[keep]] == g["expect_kept_bounds"][0]
    assert not ps.row_on[0] and not ps.col_on[j]
    red, rmap, cmap = ps.reduced()
    assert (red.m, red.n) == (lp.m - 1, lp.n - 1)
    res = PS.PresolveResult(PS.REDUCED, red, rmap, cmap, ps.records, 1, m0=lp.m, n0=lp.n)
    for a, x1, x2 in g["expect_map"]:
        x, _, _ = PS.postsolve(res, np.array([a]), np.zeros(0))
        assert list(x) == [x1, x2]


def test_doubleton_row_library_pass():
    g = load("sec2_2_doubleton_row.txt")
    lp = lp_of(g)
    pkg = capi()
    s = Library(lp, enable=pkg.LP_RULE_DOUBLETON)
    assert s.counts["doubleton"] == 1
    red = s.reduced
    assert (red.m, red.n) == (lp.m - 1, lp.n - 1)
    assert [red.col_lo[0], red.col_hi[0]] == g["expect_kept_bounds"][0]
    for a, x1, x2 in g["expect_map"]:
        x, _, _ = s.postsolve([a], [])
        assert list(x) == [x1, x2]


@pytest.mark.parametrize("side", SIDES)
def test_doubleton_row_optimum(side):
    g = load("sec2_2_doubleton_row.txt")
    s = side(lp_of(g))
    assert s.counts["doubleton"] >= 1
    x, y, _ = s.postsolve(*solve_reduced(s))
    assert list(x) == g["expect_x"][0]
    assert float(np.dot(g["c"][0], x)) == g["expect_objective"][0][0]


@pytest.mark.parametrize("side", SIDES)
def test_variable_lock(side):
    g = load("sec2_3_variable_lock.txt")
    s = side(lp_of(g))
    rule, cnt = g["expect_count"][0]
    assert s.counts[rule] == cnt
    x, _, _ = s.postsolve(*solve_reduced(s))
    assert list(x) == g["expect_x"][0]
    k = int(g["expect_unbounded_without_upper_bound"][0][0])
    hi = list(g["col_hi"][0])
    hi[k] = np.inf
    assert side(lp_of(g, col_hi=hi)).status == PS.UNBOUNDED
