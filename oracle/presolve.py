"""Oracle presolve / postsolve for eq. (1): the simple rules of Sec. 2-3.

TEST INFRASTRUCTURE ONLY (see the package header).  Plain Python loops over
dict-of-dicts row and column storage; slow, meant for small and medium LPs.

Pins (tests/test_oracle_presolve.py): the worked examples of Sec. 2 (fixing
a variable and its reduced cost, the redundant row x1 + 2 x2 >= 5 under
x1 >= 1, x2 >= 2, the doubleton x1 + x2 = 1 with x >= 0, a variable lock of
Sec. 2.3), each rule's postsolve on both signs or branches of its dual,
hand-made cases for parallel rows and columns and for propagation, and the
invariant that postsolve of an exact solution of the reduced LP (scipy's
HiGHS, independent of the oracle's PDHG) is a KKT point of the original LP
with the planted optimal objective; infeasible and unbounded LPs are
detected as such.

A reduction is a presolve transformation plus a postsolve transformation
(Sec. 2.1).  The explorers used here are the fast ones of Table 1 (empty rows
and columns, fixed columns, singleton rows, redundant rows / dominated row
sides from activity bounds, doubleton equality rows, free or implied-free
column singletons in equality rows, variable locks), run in rounds that
re-examine only what the previous round touched (Sec. 3.2).

Schedule (READING): each round runs the passes
    empty rows -> empty cols -> fixed cols -> singleton rows
    -> redundant rows / dominated sides -> doubleton equalities
    -> column singletons in inequality rows -> free column singletons
    -> variable locks,
each pass scanning its candidates in increasing index order.  Round 1 scans
every row and column; later rounds scan the rows and columns marked dirty in
the previous round.  A round in which these fast passes change nothing runs
the medium explorers of Table 1 implemented here -- primal propagation (if
asked for), dual propagation (if asked for, once), parallel rows, parallel
columns (if asked for) -- over every row
or column; the rounds stop when they find nothing either, or after 20
rounds.

Dirty marking: removing, adding or changing an entry (i, j) dirties row i and
column j; changing row bounds dirties the row; changing column bounds dirties
the column and every row holding it; changing c_j dirties column j.

Tolerances (READING): infeasibility is declared when a lower bound exceeds an
upper bound by more than 1e-9; coefficients below 1e-12 in magnitude after an
update are dropped; the rules that read the sign of a cost (empty columns,
variable locks, column singletons in inequality rows) take a cost of
magnitude at most 1e-12 * max(1, max_j |c_j| of the input LP) as zero, since
substitutions leave rounding residue (a structurally zero cost of -1e-16
would otherwise "prove" an unbounded LP).  Activity sums run over a row's entries in increasing
column order; comparisons of activities with row bounds are exact.

Variable locks (Sec. 2.3, weak dual exploration): a row i holding x_j
up-locks it when a_ij > 0 and u_i is finite or a_ij < 0 and l_i is finite,
and down-locks it in the mirrored cases.  With c_j < 0 and no up-lock every
optimal x has x_j at its upper bound (z_j < 0 for every dual feasible point),
so x_j is fixed there; with c_j > 0 and no down-lock, at its lower bound.  An
infinite target bound makes the LP unbounded (if feasible).  The fixing uses
the fixed-column reduction and its postsolve.

Column singleton in an inequality row (Table 1, dual): x_j appears only in
row i, with l_i < u_i.  Column j's dual constraint is a y_i = c_j - z_j with
z_j >= 0 when only l_j is finite, z_j <= 0 when only u_j is finite and z_j = 0
when x_j is free (a boxed x_j says nothing).  With q = c_j / a this bounds y_i
from one side; when the bound is y_i >= q > 0 (or y_i = q > 0) every optimum
has the row at its lower side, and with y_i <= q < 0 at its upper side, so the
row becomes the equality a_i x = l_i (resp. u_i) when that side is finite.
Postsolve: y_i keeps its value if it has the sign of the side it was fixed
to, else it is set to 0 (an approximate solution of the reduced problem may
put it slightly on the wrong side), with z updated over row i's entries so
that c - A^T y - z = 0 still holds.

Primal propagation (Table 1, medium; off unless asked for): in a round
where the fast passes changed nothing, before parallel rows, every row with
two or more entries is scanned in increasing index; at most 2 such sweeps
per presolve (READING: bound propagation converges slowly, each sweep
finding small further tightenings).  From its activity
bounds at the start of the row (finite contributions summed in increasing
column order, infinite ones counted; a column's "others" bound is the total
minus its own finite contribution, or the total when its own contribution is
the only infinite one), each entry a_ij x_j gets a_ij x_j >= l_i - max(others)
and a_ij x_j <= u_i - min(others) where finite.  The implied bound replaces
the column's when it is tighter by more than 1e-3 max(1, |bound|) (any finite
value of magnitude at most 1e6 replaces an infinite bound) (READING); an
implied lower bound above the upper by more than 1e-9 proves infeasibility,
one above it by less is set to the upper.  Postsolve: a reduced cost z_j
whose sign points at a tightened bound (z_j > 0 lower, z_j < 0 upper) belongs
to row i: y_i += z_j / a_ij and z_k -= a_ik z_j / a_ij over the row's entries
at that time (z_j becomes 0).

Dual propagation (Table 1, medium; off unless asked for): at a fixpoint,
after primal propagation, one sweep bounds the duals.  Every row starts with
the sign domain eq. (2) gives y_i (y_i >= 0 when only l_i is finite, <= 0 when
only u_i is, free otherwise); every column j with x_j not boxed bounds
S_j = sum_i a_ij y_i by c_j - z_j with z_j's sign domain (S_j <= c_j when only
l_j is finite, >= c_j when only u_j is, = c_j when x_j is free), and in
increasing column order each of its rows gets the bound S_j minus the other
rows' dual activity implies (activities as in primal propagation, from the
bounds at the start of the column).  Then, in increasing index, an
inequality row whose dual is at least 1e-9 becomes the equality at its
(finite) lower side, at most -1e-9 at its upper side (the reduction and
postsolve of a column singleton in an inequality row), and a column whose
reduced cost c_j - S_j is, over the final dual box, above 1e-9 max(1, |c_j|)
is fixed at its (finite) lower bound, below minus that at its upper bound
(the fixed-column reduction).  Every optimal dual lies in the box, so these
are dual reductions like variable locks (READING: one sweep, tolerance
1e-9).

Parallel columns (Table 1, medium; off unless asked for): after parallel
rows, columns with two or more entries are grouped by row pattern and, in
increasing index, column k is compared with at most 32 earlier unmerged
columns of its pattern; it is parallel to j when a_ik = s a_ij for every row
(1e-12 relative, s taken at the first row) and c_k = s c_j (1e-12 relative to
the larger of |c_k|, |s c_j|; columns whose costs are not parallel are left
alone).  Then a_j x_j + a_k x_k = a_j (x_j + s x_k): column k is removed and
x_j stands for x_j + s x_k, with bounds [l_j, u_j] + s [l_k, u_k].
Postsolve splits the merged value v: x_k = proj_[l_k,u_k](0), x_j = v - s x_k,
and if x_j leaves [l_j, u_j] it is put on the violated bound and
x_k = proj_[l_k,u_k]((v - x_j) / s); z_k = s z_j.  At an optimum where v sits
on a merged bound this puts both columns on the bounds that z's sign needs.

Parallel rows (Table 1, medium): rows k and i with the same columns and
a_k = s a_i.  Rows with two or more entries are grouped by column pattern; in
increasing index, row k is compared with the earlier rows of its pattern that
were not merged (at most 32 of them, READING) and merged into the first one
parallel to it.  Parallel means |a_kj - s a_ij| <= 1e-12 |a_kj| for every
column, with s = a_kf / a_if at the first column f (READING).  Row k's bounds,
divided by s (swapped when s < 0), are intersected with row i's; row k is
removed.  Postsolve: the merged row's y_i goes to row k as y_i / s when its
sign points at a side that came strictly from row k, otherwise it stays with
row i; the other row's y is 0.  Either way a_i y_i + a_k y_k is unchanged.

Postsolve replays the records in reverse order and keeps eq. (2)'s dual
feasibility c - A^T y - z = 0 of every intermediate problem:
  empty row / redundant row      y_i = 0
  dropped row side               nothing (y keeps a sign valid for the old row)
  fixed / empty column (value v) x_j = v,  z_j = c_j - sum_i a_ij y_i
                                 (the fix-variable postsolve of Sec. 2.1)
  singleton row a x_j in [l, u]  if z_j > 0 and the lower bound of x_j came
                                 from the row, or z_j < 0 and the upper bound
                                 did: y_i = z_j / a, z_j = 0; else y_i = 0
  doubleton a_j x_j + a_k x_k = b   x_j = (b - a_k x_k) / a_j,
                                 D_j = c_j - sum_{r != i} a_rj y_r;
                                 if the active bound of x_k (sign of z_k) was
                                 transferred from x_j: y_i = (z_k + (a_k/a_j) D_j)/a_k,
                                 z_j = D_j - a_j y_i, z_k = 0;
                                 else y_i = D_j / a_j, z_j = 0 (z_k unchanged)
  free column singleton          x_j = (b - sum_{r != j} a_ir x_r) / a_ij,
                                 y_i = c_j / a_ij, z_j = 0
  inequality made equality       y_i of the wrong sign -> 0, z_r -= a_ir dy
  parallel row k merged into i   y_k = y_i / s, y_i = 0 when y_i's sign
                                 points at a side from row k; else y_k = 0

Pins (tests/test_oracle_presolve.py): the worked examples of Sec. 2 (fixing a
variable; the redundant row x1 >= 1, x2 >= 2, x1 + 2 x2 >= 5; the doubleton
x1 + x2 = 1, x >= 0); and the invariant that postsolve of an exact solution of
the reduced problem (HiGHS) is a KKT point of the original problem whose
objective equals the planted optimum.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

FEAS_TOL = 1e-9
DROP_TOL = 1e-12
COST_TOL = 1e-12
PAR_TOL = 1e-12
PAR_CANDIDATES = 32
PROP_STEP = 1e-3
PROP_MAX_BOUND = 1e6
PROP_SWEEPS = 2
DPROP_TOL = 1e-9
MAX_ROUNDS = 20

REDUCED, INFEASIBLE, UNBOUNDED, SOLVED = 0, 1, 2, 3

INF = math.inf


@dataclass
class PresolveResult:
    status: int
    reduced: object  # a plain LP container (same attribute names as the input)
    row_map: np.ndarray  # reduced row index -> original row
    col_map: np.ndarray  # reduced col index -> original col
    records: list
    rounds: int
    counts: dict = field(default_factory=dict)
    m0: int = 0
    n0: int = 0
    seconds: float = 0.0


class _LP:
    def __init__(self, m, n, row_ptr, col_idx, val, c, off, lo, hi, lx, ux):
        self.m, self.n = m, n
        self.row_ptr, self.col_idx, self.val = row_ptr, col_idx, val
        self.c, self.obj_offset = c, off
        self.row_lo, self.row_hi, self.col_lo, self.col_hi = lo, hi, lx, ux

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


class Presolver:
    def __init__(self, lp):
        self.m, self.n = int(lp.m), int(lp.n)
        self.rows = [dict() for _ in range(self.m)]
        self.cols = [dict() for _ in range(self.n)]
        rp = np.asarray(lp.row_ptr, np.int64)
        ci = np.asarray(lp.col_idx, np.int64)
        va = np.asarray(lp.val, np.float64)
        for i in range(self.m):
            for k in range(int(rp[i]), int(rp[i + 1])):
                j = int(ci[k])
                v = float(va[k])
                if v != 0.0:
                    self.rows[i][j] = v
                    self.cols[j][i] = v
        self.c = [float(v) for v in lp.c]
        self.cost_tol = COST_TOL * max([1.0] + [abs(v) for v in self.c])
        self.off = float(lp.obj_offset)
        self.lo = [float(v) for v in lp.row_lo]
        self.hi = [float(v) for v in lp.row_hi]
        self.lx = [float(v) for v in lp.col_lo]
        self.ux = [float(v) for v in lp.col_hi]
        self.row_on = [True] * self.m
        self.col_on = [True] * self.n
        self.records = []
        self.dirty_r = set()
        self.dirty_c = set()
        self.changed = False
        self.status = REDUCED
        self.counts = {k: 0 for k in ("empty_row", "empty_col", "fixed_col", "singleton_row",
                                      "redundant_row", "dropped_side", "doubleton",
                                      "free_col_singleton", "dual_fix", "ineq_to_eq",
                                      "parallel_row", "tightened", "parallel_col",
                                      "dual_prop")}

    # -- primitive edits with dirty marking --------------------------------
    def _mark_col_bounds(self, j):
        self.dirty_c.add(j)
        for i in self.cols[j]:
            self.dirty_r.add(i)

    def _remove_entry(self, i, j):
        del self.rows[i][j]
        del self.cols[j][i]
        self.dirty_r.add(i)
        self.dirty_c.add(j)

    def _set_entry(self, i, j, v):
        if abs(v) < DROP_TOL:
            if j in self.rows[i]:
                self._remove_entry(i, j)
            return
        self.rows[i][j] = v
        self.cols[j][i] = v
        self.dirty_r.add(i)
        self.dirty_c.add(j)

    def _remove_row(self, i):
        for j in list(self.rows[i].keys()):
            self._remove_entry(i, j)
        self.row_on[i] = False

    def _remove_col(self, j):
        for i in list(self.cols[j].keys()):
            self._remove_entry(i, j)
        self.col_on[j] = False

    def _activity(self, i, skip=-1):
        """(min, max) of sum_j a_ij x_j over the column bounds, ascending j."""
        lo_s = 0.0
        hi_s = 0.0
        lo_inf = 0
        hi_inf = 0
        for j in sorted(self.rows[i]):
            if j == skip:
                continue
            a = self.rows[i][j]
            if a > 0:
                bl, bu = self.lx[j], self.ux[j]
            else:
                bl, bu = self.ux[j], self.lx[j]
            if math.isinf(bl):
                lo_inf += 1
            else:
                lo_s += a * bl
            if math.isinf(bu):
                hi_inf += 1
            else:
                hi_s += a * bu
        return (-INF if lo_inf else lo_s), (INF if hi_inf else hi_s)

    # -- rules ---------------------------------------------------------------
    def empty_row(self, i):
        if self.lo[i] > FEAS_TOL or self.hi[i] < -FEAS_TOL:
            self.status = INFEASIBLE
            return
        self.records.append(("empty_row", i))
        self.row_on[i] = False
        self.counts["empty_row"] += 1
        self.changed = True

    def empty_col(self, j):
        cj = self.c[j]
        if cj > self.cost_tol:
            v = self.lx[j]
        elif cj < -self.cost_tol:
            v = self.ux[j]
        else:
            v = min(max(0.0, self.lx[j]), self.ux[j])
        if math.isinf(v):
            self.status = UNBOUNDED
            return
        self.off += cj * v
        self.records.append(("fix_col", j, v, cj, []))
        self.col_on[j] = False
        self.dirty_c.add(j)
        self.counts["empty_col"] += 1
        self.changed = True

    def fixed_col(self, j):
        v = self.lx[j]
        entries = sorted(self.cols[j].items())
        for i, a in entries:
            if not math.isinf(self.lo[i]):
                self.lo[i] -= a * v
            if not math.isinf(self.hi[i]):
                self.hi[i] -= a * v
            self.dirty_r.add(i)
        self.off += self.c[j] * v
        self.records.append(("fix_col", j, v, self.c[j], entries))
        self._remove_col(j)
        self.counts["fixed_col"] += 1
        self.changed = True

    def singleton_row(self, i):
        (j, a), = self.rows[i].items()
        if a > 0:
            ilo = self.lo[i] / a if not math.isinf(self.lo[i]) else -INF
            ihi = self.hi[i] / a if not math.isinf(self.hi[i]) else INF
        else:
            ilo = self.hi[i] / a if not math.isinf(self.hi[i]) else -INF
            ihi = self.lo[i] / a if not math.isinf(self.lo[i]) else INF
        lo_from = ilo > self.lx[j]
        hi_from = ihi < self.ux[j]
        nl = ilo if lo_from else self.lx[j]
        nu = ihi if hi_from else self.ux[j]
        if nl > nu + FEAS_TOL:
            self.status = INFEASIBLE
            return
        if nl > nu:
            nl = nu = 0.5 * (nl + nu)
        self.records.append(("singleton_row", i, j, a, lo_from, hi_from))
        self._remove_row(i)
        if nl != self.lx[j] or nu != self.ux[j]:
            self.lx[j] = nl
            self.ux[j] = nu
            self._mark_col_bounds(j)
        self.counts["singleton_row"] += 1
        self.changed = True

    def redundant_row(self, i):
        lo, hi = self.lo[i], self.hi[i]
        if lo == hi:
            return
        amin, amax = self._activity(i)
        lo_imp = math.isinf(lo) or amin >= lo
        hi_imp = math.isinf(hi) or amax <= hi
        if lo_imp and hi_imp:
            self.records.append(("redundant_row", i))
            self._remove_row(i)
            self.counts["redundant_row"] += 1
            self.changed = True
        elif lo_imp and not math.isinf(lo):
            self.records.append(("drop_side", i, 0, lo))
            self.lo[i] = -INF
            self.dirty_r.add(i)
            self.counts["dropped_side"] += 1
            self.changed = True
        elif hi_imp and not math.isinf(hi):
            self.records.append(("drop_side", i, 1, hi))
            self.hi[i] = INF
            self.dirty_r.add(i)
            self.counts["dropped_side"] += 1
            self.changed = True

    def doubleton(self, i):
        (p, ap), (q, aq) = sorted(self.rows[i].items())
        b = self.lo[i]
        # eliminate the larger |a| (so |a_k / a_j| <= 1); ties: fewer column
        # entries, then lower index
        if abs(ap) > abs(aq):
            j, aj, k, ak = p, ap, q, aq
        elif abs(aq) > abs(ap):
            j, aj, k, ak = q, aq, p, ap
        elif len(self.cols[q]) < len(self.cols[p]):
            j, aj, k, ak = q, aq, p, ap
        else:
            j, aj, k, ak = p, ap, q, aq
        r = ak / aj
        s = b / aj
        # l_j <= s - r x_k <= u_j  ->  r x_k in [s - u_j, s - l_j]
        t_lo = s - self.ux[j] if not math.isinf(self.ux[j]) else -INF
        t_hi = s - self.lx[j] if not math.isinf(self.lx[j]) else INF
        if r > 0:
            ilo = t_lo / r if not math.isinf(t_lo) else -INF
            ihi = t_hi / r if not math.isinf(t_hi) else INF
        else:
            ilo = t_hi / r if not math.isinf(t_hi) else -INF
            ihi = t_lo / r if not math.isinf(t_lo) else INF
        lo_from = ilo > self.lx[k]
        hi_from = ihi < self.ux[k]
        nl = ilo if lo_from else self.lx[k]
        nu = ihi if hi_from else self.ux[k]
        if nl > nu + FEAS_TOL:
            self.status = INFEASIBLE
            return
        if nl > nu:
            nl = nu = 0.5 * (nl + nu)
        colj = sorted((rr, a) for rr, a in self.cols[j].items() if rr != i)
        cj = self.c[j]
        self.records.append(("doubleton", i, j, k, aj, ak, b, cj, lo_from, hi_from, colj))
        # objective: c_j x_j = c_j s - c_j r x_k
        self.off += cj * s
        if cj != 0.0:
            self.c[k] -= cj * r
            self.dirty_c.add(k)
        # substitute into the other rows of column j
        for rr, a in colj:
            if not math.isinf(self.lo[rr]):
                self.lo[rr] -= a * s
            if not math.isinf(self.hi[rr]):
                self.hi[rr] -= a * s
            old = self.rows[rr].get(k, 0.0)
            self._remove_entry(rr, j)
            self._set_entry(rr, k, old - a * r)
        self._remove_row(i)
        self._remove_col(j)
        if nl != self.lx[k] or nu != self.ux[k]:
            self.lx[k] = nl
            self.ux[k] = nu
            self._mark_col_bounds(k)
        self.counts["doubleton"] += 1
        self.changed = True

    def free_col_singleton(self, j):
        (i, a), = self.cols[j].items()
        if not self.row_on[i] or self.lo[i] != self.hi[i] or len(self.rows[i]) < 2:
            return
        b = self.lo[i]
        free = math.isinf(self.lx[j]) and math.isinf(self.ux[j])
        if not free:
            amin, amax = self._activity(i, skip=j)
            if a > 0:
                ilo, ihi = (b - amax) / a, (b - amin) / a
            else:
                ilo, ihi = (b - amin) / a, (b - amax) / a
            if not (ilo >= self.lx[j] and ihi <= self.ux[j]):
                return
        cj = self.c[j]
        others = sorted((r, v) for r, v in self.rows[i].items() if r != j)
        self.records.append(("free_col_singleton", i, j, a, b, cj, others))
        self.off += cj * b / a
        if cj != 0.0:
            for r, v in others:
                self.c[r] -= cj * v / a
                self.dirty_c.add(r)
        self._remove_row(i)
        self._remove_col(j)
        self.counts["free_col_singleton"] += 1
        self.changed = True

    def locks(self, j):
        """(up-locked, down-locked) of column j from its rows' finite bounds"""
        up = down = False
        for i, a in self.cols[j].items():
            lf = not math.isinf(self.lo[i])
            uf = not math.isinf(self.hi[i])
            if a > 0:
                up = up or uf
                down = down or lf
            else:
                up = up or lf
                down = down or uf
        return up, down

    def dual_fix(self, j):
        cj = self.c[j]
        if abs(cj) <= self.cost_tol:
            return
        up, down = self.locks(j)
        if cj < 0 and not up:
            v = self.ux[j]
        elif cj > 0 and not down:
            v = self.lx[j]
        else:
            return
        if math.isinf(v):
            self.status = UNBOUNDED
            return
        self.lx[j] = v
        self.ux[j] = v
        self.fixed_col(j)
        self.counts["fixed_col"] -= 1
        self.counts["dual_fix"] += 1

    def col_singleton_ineq(self, j):
        (i, a), = self.cols[j].items()
        lo, hi = self.lo[i], self.hi[i]
        if lo == hi:
            return
        lf = not math.isinf(self.lx[j])
        uf = not math.isinf(self.ux[j])
        if (lf and uf) or abs(self.c[j]) <= self.cost_tol:
            return
        # a y_i = c_j - z_j with z_j >= 0 (only l_j finite), <= 0 (only u_j
        # finite) or = 0 (free): the side of q = c_j / a that y_i must lie on
        if lf:
            y_ge_q, y_le_q = a < 0, a > 0
        elif uf:
            y_ge_q, y_le_q = a > 0, a < 0
        else:
            y_ge_q = y_le_q = True
        q = self.c[j] / a
        if y_ge_q and q > 0 and not math.isinf(lo):
            side = 1
            self.hi[i] = lo
        elif y_le_q and q < 0 and not math.isinf(hi):
            side = -1
            self.lo[i] = hi
        else:
            return
        self.records.append(("row_to_eq", i, side, sorted(self.rows[i].items())))
        self.dirty_r.add(i)
        self.counts["ineq_to_eq"] += 1
        self.changed = True

    def _parallel_scale(self, i, k):
        """s with a_k = s a_i (to PAR_TOL), or None; same column pattern."""
        ri, rk = self.rows[i], self.rows[k]
        f = min(ri)
        s = rk[f] / ri[f]
        for j, a in ri.items():
            if abs(rk[j] - s * a) > PAR_TOL * abs(rk[j]):
                return None
        return s

    def merge_parallel(self, i, k, s):
        lk, uk = self.lo[k], self.hi[k]
        if s > 0:
            nlk = -INF if math.isinf(lk) else lk / s
            nuk = INF if math.isinf(uk) else uk / s
        else:
            nlk = -INF if math.isinf(uk) else uk / s
            nuk = INF if math.isinf(lk) else lk / s
        lo_from = nlk > self.lo[i]
        hi_from = nuk < self.hi[i]
        nl = nlk if lo_from else self.lo[i]
        nu = nuk if hi_from else self.hi[i]
        if nl > nu + FEAS_TOL:
            self.status = INFEASIBLE
            return
        if nl > nu:
            nl = nu = 0.5 * (nl + nu)
        self.records.append(("parallel_row", i, k, s, lo_from, hi_from))
        self._remove_row(k)
        if nl != self.lo[i] or nu != self.hi[i]:
            self.lo[i] = nl
            self.hi[i] = nu
            self.dirty_r.add(i)
        self.counts["parallel_row"] += 1
        self.changed = True

    def _row_sums(self, i):
        """finite min / max activity sums over ascending columns and the
        counts of infinite contributions"""
        smin = smax = 0.0
        nmin = nmax = 0
        for j in sorted(self.rows[i]):
            a = self.rows[i][j]
            bl, bu = (self.lx[j], self.ux[j]) if a > 0 else (self.ux[j], self.lx[j])
            if math.isinf(bl):
                nmin += 1
            else:
                smin += a * bl
            if math.isinf(bu):
                nmax += 1
            else:
                smax += a * bu
        return smin, nmin, smax, nmax

    def _better(self, new, old, lower):
        if math.isinf(new):
            return False
        if math.isinf(old):
            return abs(new) <= PROP_MAX_BOUND
        step = PROP_STEP * max(1.0, abs(old))
        return new > old + step if lower else new < old - step

    def propagate_row(self, i):
        lo, hi = self.lo[i], self.hi[i]
        smin, nmin, smax, nmax = self._row_sums(i)
        ents = sorted(self.rows[i].items())
        found = []
        for j, a in ents:
            bl, bu = (self.lx[j], self.ux[j]) if a > 0 else (self.ux[j], self.lx[j])
            if math.isinf(bu):
                omax = smax if nmax == 1 else INF
            else:
                omax = smax - a * bu if nmax == 0 else INF
            if math.isinf(bl):
                omin = smin if nmin == 1 else -INF
            else:
                omin = smin - a * bl if nmin == 0 else -INF
            t_lo = lo - omax if not (math.isinf(lo) or math.isinf(omax)) else -INF  # a x_j >= t_lo
            t_hi = hi - omin if not (math.isinf(hi) or math.isinf(omin)) else INF   # a x_j <= t_hi
            if a > 0:
                nl = t_lo / a if not math.isinf(t_lo) else -INF
                nu = t_hi / a if not math.isinf(t_hi) else INF
            else:
                nl = t_hi / a if not math.isinf(t_hi) else -INF
                nu = t_lo / a if not math.isinf(t_lo) else INF
            found.append((j, a, nl, nu))
        for j, a, nl, nu in found:
            for side, new in ((0, nl), (1, nu)):
                old = self.lx[j] if side == 0 else self.ux[j]
                if not self._better(new, old, side == 0):
                    continue
                other = self.ux[j] if side == 0 else self.lx[j]
                if (new > other + FEAS_TOL) if side == 0 else (new < other - FEAS_TOL):
                    self.status = INFEASIBLE
                    return
                if (new > other) if side == 0 else (new < other):
                    new = other
                self.records.append(("tighten", j, i, a, side, ents))
                if side == 0:
                    self.lx[j] = new
                else:
                    self.ux[j] = new
                self._mark_col_bounds(j)
                self.counts["tightened"] += 1
                self.changed = True

    def propagate(self):
        for i in range(self.m):
            if self.row_on[i] and len(self.rows[i]) >= 2:
                self.propagate_row(i)
                if self.status != REDUCED:
                    return

    @staticmethod
    def _range_sums(terms):
        """finite sums of the lower / upper ends of a list of (lo, hi)
        contributions and the counts of infinite ones"""
        slo = shi = 0.0
        nlo = nhi = 0
        for lo, hi in terms:
            if math.isinf(lo):
                nlo += 1
            else:
                slo += lo
            if math.isinf(hi):
                nhi += 1
            else:
                shi += hi
        return slo, nlo, shi, nhi

    @staticmethod
    def _scaled_range(a, lo, hi):
        """range of a * y for y in [lo, hi]"""
        if a > 0:
            return (a * lo if not math.isinf(lo) else -INF, a * hi if not math.isinf(hi) else INF)
        return (a * hi if not math.isinf(hi) else -INF, a * lo if not math.isinf(lo) else INF)

    def dual_propagate(self):
        yl, yu = {}, {}
        for i in range(self.m):
            if self.row_on[i]:
                yl[i] = 0.0 if math.isinf(self.hi[i]) else -INF
                yu[i] = 0.0 if math.isinf(self.lo[i]) else INF
        for j in range(self.n):
            if not self.col_on[j] or not self.cols[j]:
                continue
            lf, uf = not math.isinf(self.lx[j]), not math.isinf(self.ux[j])
            if lf and uf:
                continue
            cj = self.c[j]
            dl = -INF if lf else cj
            du = INF if uf else cj
            ents = sorted(self.cols[j].items())
            terms = [self._scaled_range(a, yl[i], yu[i]) for i, a in ents]
            slo, nlo, shi, nhi = self._range_sums(terms)
            found = []
            for (i, a), (tlo, thi) in zip(ents, terms):
                if math.isinf(thi):
                    omax = shi if nhi == 1 else INF
                else:
                    omax = shi - thi if nhi == 0 else INF
                if math.isinf(tlo):
                    omin = slo if nlo == 1 else -INF
                else:
                    omin = slo - tlo if nlo == 0 else -INF
                # a y_i in [dl - omax, du - omin]
                t_lo = dl - omax if not (math.isinf(dl) or math.isinf(omax)) else -INF
                t_hi = du - omin if not (math.isinf(du) or math.isinf(omin)) else INF
                if a > 0:
                    nl = t_lo / a if not math.isinf(t_lo) else -INF
                    nu = t_hi / a if not math.isinf(t_hi) else INF
                else:
                    nl = t_hi / a if not math.isinf(t_hi) else -INF
                    nu = t_lo / a if not math.isinf(t_lo) else INF
                found.append((i, nl, nu))
            for i, nl, nu in found:
                if nl > yl[i]:
                    yl[i] = nl
                if nu < yu[i]:
                    yu[i] = nu
        for i in range(self.m):
            if not self.row_on[i] or self.lo[i] == self.hi[i] or not self.rows[i]:
                continue
            if yl[i] >= DPROP_TOL and not math.isinf(self.lo[i]):
                side = 1
                self.hi[i] = self.lo[i]
            elif yu[i] <= -DPROP_TOL and not math.isinf(self.hi[i]):
                side = -1
                self.lo[i] = self.hi[i]
            else:
                continue
            self.records.append(("row_to_eq", i, side, sorted(self.rows[i].items())))
            self.dirty_r.add(i)
            self.counts["dual_prop"] += 1
            self.changed = True
        for j in range(self.n):
            if not self.col_on[j] or not self.cols[j] or self.lx[j] == self.ux[j]:
                continue
            terms = [self._scaled_range(a, yl[i], yu[i]) for i, a in sorted(self.cols[j].items())]
            slo, nlo, shi, nhi = self._range_sums(terms)
            cj = self.c[j]
            tol = DPROP_TOL * max(1.0, abs(cj))
            zmin = cj - shi if nhi == 0 else -INF
            zmax = cj - slo if nlo == 0 else INF
            if zmin > tol and not math.isinf(self.lx[j]):
                v = self.lx[j]
            elif zmax < -tol and not math.isinf(self.ux[j]):
                v = self.ux[j]
            else:
                continue
            self.lx[j] = v
            self.ux[j] = v
            self.fixed_col(j)
            self.counts["fixed_col"] -= 1
            self.counts["dual_prop"] += 1

    def parallel_rows(self):
        reps = {}  # column pattern -> rows not merged, increasing index
        for k in range(self.m):
            if not self.row_on[k] or len(self.rows[k]) < 2:
                continue
            key = tuple(sorted(self.rows[k]))
            lst = reps.setdefault(key, [])
            for i in lst[:PAR_CANDIDATES]:
                s = self._parallel_scale(i, k)
                if s is not None:
                    self.merge_parallel(i, k, s)
                    if self.status != REDUCED:
                        return
                    break
            else:
                lst.append(k)

    def _parallel_col_scale(self, j, k):
        """s with a_k = s a_j and c_k = s c_j (to PAR_TOL), or None"""
        cj, ck = self.cols[j], self.cols[k]
        f = min(cj)
        s = ck[f] / cj[f]
        for i, a in cj.items():
            if abs(ck[i] - s * a) > PAR_TOL * abs(ck[i]):
                return None
        sc = s * self.c[j]
        if abs(self.c[k] - sc) > PAR_TOL * max(abs(self.c[k]), abs(sc)):
            return None
        return s

    def merge_parallel_col(self, j, k, s):
        lj, uj, lk, uk = self.lx[j], self.ux[j], self.lx[k], self.ux[k]
        if s > 0:
            nl, nu = lj + s * lk, uj + s * uk
        else:
            nl, nu = lj + s * uk, uj + s * lk
        self.records.append(("parallel_col", j, k, s, lj, uj, lk, uk))
        self._remove_col(k)
        self.lx[j] = nl
        self.ux[j] = nu
        self._mark_col_bounds(j)
        self.counts["parallel_col"] += 1
        self.changed = True

    def parallel_cols(self):
        reps = {}  # row pattern -> columns not merged, increasing index
        for k in range(self.n):
            if not self.col_on[k] or len(self.cols[k]) < 2:
                continue
            key = tuple(sorted(self.cols[k]))
            lst = reps.setdefault(key, [])
            for j in lst[:PAR_CANDIDATES]:
                s = self._parallel_col_scale(j, k)
                if s is not None:
                    self.merge_parallel_col(j, k, s)
                    break
            else:
                lst.append(k)

    # -- driver ----------------------------------------------------------------
    def run(self, max_rounds=MAX_ROUNDS, propagation=False, parallel_cols=False,
            dual_propagation=False):
        sweeps = 0
        dsweeps = 0
        rows_c = list(range(self.m))
        cols_c = list(range(self.n))
        rounds = 0
        for rnd in range(max_rounds):
            rounds = rnd + 1
            self.dirty_r = set()
            self.dirty_c = set()
            self.changed = False
            for i in rows_c:
                if self.row_on[i] and not self.rows[i]:
                    self.empty_row(i)
                    if self.status != REDUCED:
                        return rounds
            for j in cols_c:
                if self.col_on[j] and not self.cols[j]:
                    self.empty_col(j)
                    if self.status != REDUCED:
                        return rounds
            for j in cols_c:
                if self.col_on[j] and self.lx[j] == self.ux[j]:
                    self.fixed_col(j)
            for i in rows_c:
                if self.row_on[i] and len(self.rows[i]) == 1:
                    self.singleton_row(i)
                    if self.status != REDUCED:
                        return rounds
            for i in rows_c:
                if self.row_on[i] and len(self.rows[i]) >= 1:
                    self.redundant_row(i)
            for i in rows_c:
                if (self.row_on[i] and len(self.rows[i]) == 2
                        and self.lo[i] == self.hi[i]):
                    self.doubleton(i)
                    if self.status != REDUCED:
                        return rounds
            for j in cols_c:
                if self.col_on[j] and len(self.cols[j]) == 1:
                    self.col_singleton_ineq(j)
            for j in cols_c:
                if self.col_on[j] and len(self.cols[j]) == 1:
                    self.free_col_singleton(j)
            for j in cols_c:
                if self.col_on[j] and self.cols[j]:
                    self.dual_fix(j)
                    if self.status != REDUCED:
                        return rounds
            if not self.changed:
                if propagation and sweeps < PROP_SWEEPS:
                    sweeps += 1
                    self.propagate()
                    if self.status != REDUCED:
                        return rounds
                if dual_propagation and dsweeps < 1:
                    dsweeps += 1
                    self.dual_propagate()
                self.parallel_rows()
                if parallel_cols and self.status == REDUCED:
                    self.parallel_cols()
                if self.status != REDUCED:
                    return rounds
                if not self.changed:
                    break
            rows_c = sorted(i for i in self.dirty_r if self.row_on[i])
            cols_c = sorted(j for j in self.dirty_c if self.col_on[j])
        return rounds

    def reduced(self):
        rmap = np.array([i for i in range(self.m) if self.row_on[i]], dtype=np.int64)
        cmap = np.array([j for j in range(self.n) if self.col_on[j]], dtype=np.int64)
        cpos = -np.ones(self.n, dtype=np.int64)
        cpos[cmap] = np.arange(cmap.shape[0])
        rp = [0]
        ci = []
        va = []
        for i in rmap:
            for j in sorted(self.rows[i]):
                ci.append(cpos[j])
                va.append(self.rows[i][j])
            rp.append(len(ci))
        lp = _LP(int(rmap.shape[0]), int(cmap.shape[0]), np.array(rp, dtype=np.int64),
                 np.array(ci, dtype=np.int32), np.array(va, dtype=np.float64),
                 np.array([self.c[j] for j in cmap], dtype=np.float64), self.off,
                 np.array([self.lo[i] for i in rmap], dtype=np.float64),
                 np.array([self.hi[i] for i in rmap], dtype=np.float64),
                 np.array([self.lx[j] for j in cmap], dtype=np.float64),
                 np.array([self.ux[j] for j in cmap], dtype=np.float64))
        return lp, rmap, cmap


def presolve(lp, max_rounds: int = MAX_ROUNDS, propagation: bool = False,
             parallel_cols: bool = False, dual_propagation: bool = False) -> PresolveResult:
    t0 = time.perf_counter()
    ps = Presolver(lp)
    rounds = ps.run(max_rounds, propagation, parallel_cols, dual_propagation)
    red, rmap, cmap = ps.reduced()
    status = ps.status
    if status == REDUCED and red.m == 0 and red.n == 0:
        status = SOLVED
    return PresolveResult(status=status, reduced=red, row_map=rmap, col_map=cmap,
                          records=ps.records, rounds=rounds, counts=ps.counts,
                          m0=ps.m, n0=ps.n, seconds=time.perf_counter() - t0)


def postsolve(res: PresolveResult, x_red, y_red, z_red=None):
    """Map a (approximate) solution of the reduced LP to (x, y, z) of the
    original LP by replaying the postsolve records in reverse."""
    x = np.zeros(res.n0)
    y = np.zeros(res.m0)
    z = np.zeros(res.n0)
    red = res.reduced
    x[res.col_map] = x_red
    y[res.row_map] = y_red
    if z_red is None:
        A = _csr(red)
        z_red = np.asarray(red.c, np.float64) - A.T @ np.asarray(y_red, np.float64)
    z[res.col_map] = z_red
    for rec in reversed(res.records):
        kind = rec[0]
        if kind in ("empty_row", "redundant_row"):
            y[rec[1]] = 0.0
        elif kind == "drop_side":
            pass
        elif kind == "fix_col":
            _, j, v, cj, entries = rec
            x[j] = v
            s = cj
            for i, a in entries:
                s -= a * y[i]
            z[j] = s
        elif kind == "singleton_row":
            _, i, j, a, lo_from, hi_from = rec
            if (z[j] > 0 and lo_from) or (z[j] < 0 and hi_from):
                y[i] = z[j] / a
                z[j] = 0.0
            else:
                y[i] = 0.0
        elif kind == "doubleton":
            _, i, j, k, aj, ak, b, cj, lo_from, hi_from, colj = rec
            x[j] = (b - ak * x[k]) / aj
            dj = cj
            for rr, a in colj:
                dj -= a * y[rr]
            if (z[k] > 0 and lo_from) or (z[k] < 0 and hi_from):
                y[i] = (z[k] + (ak / aj) * dj) / ak
                z[j] = dj - aj * y[i]
                z[k] = 0.0
            else:
                y[i] = dj / aj
                z[j] = 0.0
        elif kind == "row_to_eq":
            _, i, side, entries = rec
            if (side > 0 and y[i] < 0) or (side < 0 and y[i] > 0):
                d = -y[i]
                y[i] = 0.0
                for k, a in entries:
                    z[k] -= a * d
        elif kind == "tighten":
            _, j, i, a, side, entries = rec
            if (side == 0 and z[j] > 0) or (side == 1 and z[j] < 0):
                d = z[j] / a
                y[i] += d
                for k, ak in entries:
                    z[k] -= ak * d
                z[j] = 0.0
        elif kind == "parallel_col":
            _, j, k, s, lj, uj, lk, uk = rec
            v = x[j]
            xk = min(max(0.0, lk), uk)
            xj = v - s * xk
            if xj < lj:
                xj = lj
                xk = min(max((v - xj) / s, lk), uk)
            elif xj > uj:
                xj = uj
                xk = min(max((v - xj) / s, lk), uk)
            x[j] = xj
            x[k] = xk
            z[k] = s * z[j]
        elif kind == "parallel_row":
            _, i, k, s, lo_from, hi_from = rec
            if (y[i] > 0 and lo_from) or (y[i] < 0 and hi_from):
                y[k] = y[i] / s
                y[i] = 0.0
            else:
                y[k] = 0.0
        elif kind == "free_col_singleton":
            _, i, j, a, b, cj, others = rec
            s = b
            for r, v in others:
                s -= v * x[r]
            x[j] = s / a
            y[i] = cj / a
            z[j] = 0.0
        else:  # pragma: no cover
            raise ValueError(kind)
    return x, y, z


def _csr(lp):
    import scipy.sparse as sp

    return sp.csr_matrix((np.asarray(lp.val, np.float64), np.asarray(lp.col_idx, np.int64),
                          np.asarray(lp.row_ptr, np.int64)), shape=(lp.m, lp.n))
