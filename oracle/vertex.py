"""Brute-force optimum of a tiny bounded LP by vertex enumeration.

TEST INFRASTRUCTURE ONLY.  The optimum of eq. (1) with every column bounded
and a nonempty feasible set is attained at a vertex: a point where n linearly
independent constraint hyperplanes (row sides a_i x = l_i / u_i and bound
sides x_j = l_j / u_j) are active.  Enumerate every n-subset, solve, keep the
feasible points, take the minimum of c^T x.  Exponential; for n <= 6, m <= 5.
"""
from __future__ import annotations

import itertools

import numpy as np


def vertex_optimum(lp, tol: float = 1e-9):
    """Return (p*, x*) by enumeration; p* includes the objective offset."""
    m, n = lp.m, lp.n
    A = np.zeros((m, n))
    for i in range(m):
        for k in range(int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])):
            A[i, int(lp.col_idx[k])] = lp.val[k]
    lo_r, hi_r = np.asarray(lp.row_lo, float), np.asarray(lp.row_hi, float)
    lo_x, hi_x = np.asarray(lp.col_lo, float), np.asarray(lp.col_hi, float)
    if not (np.all(np.isfinite(lo_x)) and np.all(np.isfinite(hi_x))):
        raise ValueError("vertex enumeration needs finite column bounds")
    planes = []  # (normal, rhs)
    for i in range(m):
        if np.isfinite(lo_r[i]):
            planes.append((A[i], lo_r[i]))
        if np.isfinite(hi_r[i]) and hi_r[i] != lo_r[i]:
            planes.append((A[i], hi_r[i]))
    eye = np.eye(n)
    for j in range(n):
        planes.append((eye[j], lo_x[j]))
        if hi_x[j] != lo_x[j]:
            planes.append((eye[j], hi_x[j]))
    N = np.array([p[0] for p in planes])
    b = np.array([p[1] for p in planes])
    combos = np.array(list(itertools.combinations(range(len(planes)), n)), dtype=np.int64)
    M = N[combos]  # (C, n, n)
    rhs = b[combos]
    det = np.linalg.det(M)
    ok = np.abs(det) > 1e-10
    X = np.linalg.solve(M[ok], rhs[ok][..., None])[..., 0]
    ax = X @ A.T
    feas = (
        np.all(X >= lo_x - tol, axis=1) & np.all(X <= hi_x + tol, axis=1)
        & np.all(ax >= lo_r - tol, axis=1) & np.all(ax <= hi_r + tol, axis=1)
    )
    if not feas.any():
        raise ValueError("no feasible vertex")
    obj = X[feas] @ np.asarray(lp.c, float)
    best = int(np.argmin(obj))
    return float(obj[best]) + float(lp.obj_offset), X[feas][best]
