"""Small LPs without an optimum (test inputs shared by the oracle and GPU
tests): primal infeasible and unbounded, tiny and random."""
import numpy as np

import lpgen
from lp_helpers import SimpleLP

INF = np.inf


def tiny_infeasible():
    # x >= 0 and x1 + x2 <= -1
    return SimpleLP([[1.0, 1.0], [1.0, -1.0]], [1.0, 1.0], [-INF, -2.0], [-1.0, 2.0],
                    [0.0, 0.0], [INF, INF])


def tiny_unbounded():
    # min -x1 - x2 with -1 <= x1 - x2 <= 1, x >= 0: the ray (1, 1)
    return SimpleLP([[1.0, -1.0]], [-1.0, -1.0], [-1.0], [1.0], [0.0, 0.0], [INF, INF])


def random_infeasible(seed=0, m=30, n=60):
    # A >= 0, x >= 0 and A x = b with one b_i < 0
    rng = np.random.default_rng(seed)
    A = (rng.random((m, n)) < 0.2) * rng.uniform(0.5, 2.0, (m, n))
    A[np.arange(m), rng.integers(0, n, m)] += 1.0
    b = A @ rng.uniform(0.0, 1.0, n)
    b[3] = -0.5
    return SimpleLP(A, rng.normal(size=n), b, b, np.zeros(n), np.full(n, INF))


def random_unbounded():
    # the planted C1 LP plus two columns x_a - x_b in row 0 with negative
    # costs: the ray e_a + e_b keeps every row and lowers the cost
    lp = lpgen.c1_small()
    A = lp.csr().toarray()
    extra = np.zeros((lp.m, 2))
    extra[0, 0], extra[0, 1] = 1.0, -1.0
    return SimpleLP(np.hstack([A, extra]), np.concatenate([lp.c, [-1.0, -0.5]]), lp.row_lo,
                    lp.row_hi, np.concatenate([lp.col_lo, [0.0, 0.0]]),
                    np.concatenate([lp.col_hi, [INF, INF]]))


CASES = [("tiny_infeasible", tiny_infeasible, 4), ("tiny_unbounded", tiny_unbounded, 5),
         ("random_infeasible", random_infeasible, 4), ("random_unbounded", random_unbounded, 5)]
