"""Test-side helpers: conversions to scipy's linprog form and small LPs."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


class SimpleLP:
    """Plain container with the attribute names both sides accept."""

    def __init__(self, A, c, row_lo, row_hi, col_lo, col_hi, obj_offset=0.0):
        A = sp.csr_matrix(A, dtype=np.float64)
        A.sort_indices()
        self.m, self.n = A.shape
        self.row_ptr = A.indptr.astype(np.int64)
        self.col_idx = A.indices.astype(np.int32)
        self.val = A.data.astype(np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.row_lo = np.asarray(row_lo, dtype=np.float64)
        self.row_hi = np.asarray(row_hi, dtype=np.float64)
        self.col_lo = np.asarray(col_lo, dtype=np.float64)
        self.col_hi = np.asarray(col_hi, dtype=np.float64)
        self.obj_offset = float(obj_offset)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def csr(self):
        return sp.csr_matrix((self.val, self.col_idx.astype(np.int64), self.row_ptr),
                             shape=(self.m, self.n))


def csr(lp):
    return sp.csr_matrix((np.asarray(lp.val, float), np.asarray(lp.col_idx, np.int64),
                          np.asarray(lp.row_ptr, np.int64)), shape=(lp.m, lp.n))


def highs_solve(lp):
    """Solve with scipy's HiGHS; return (objective incl. offset, x, y) where y
    follows eq. (2)'s sign convention (y > 0 on an active lower side)."""
    A = csr(lp)
    lo, hi = np.asarray(lp.row_lo, float), np.asarray(lp.row_hi, float)
    eq = np.isfinite(lo) & np.isfinite(hi) & (lo == hi)
    up = np.isfinite(hi) & ~eq
    dn = np.isfinite(lo) & ~eq
    A_ub = sp.vstack([A[up], -A[dn]]).tocsr()
    b_ub = np.concatenate([hi[up], -lo[dn]])
    kw = {}
    if A_ub.shape[0]:
        kw.update(A_ub=A_ub, b_ub=b_ub)
    if eq.any():
        kw.update(A_eq=A[eq], b_eq=lo[eq])
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lp.col_lo, lp.col_hi)]
    res = linprog(lp.c, bounds=bounds, method="highs", **kw)
    assert res.status == 0, res.message
    y = np.zeros(lp.m)
    if eq.any():
        y[eq] = res.eqlin.marginals
    if A_ub.shape[0]:
        mu = res.ineqlin.marginals
        nu = int(up.sum())
        y[up] += mu[:nu]
        y[dn] -= mu[nu:]
    return float(res.fun) + float(lp.obj_offset), res.x, y
