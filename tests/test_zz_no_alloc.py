"""The allocation-free power-iteration entry point (lp_power_norm_static).

It is for callers that cannot allocate device memory where they need the
step-size estimate (a process that reserved the GPU for its own pool, a
latency-critical path that must not call cudaMalloc).  The GPU test checks
it against the step size the allocating path (lp_solve) reports, on two
calls in a row; this file is collected last so a failure here comes after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import lpgen


def _lib():
    import paper_2604_23951_gb300 as pkg

    try:
        return pkg, pkg.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def test_rejects_sizes_beyond_the_static_scratch():
    pkg, lib = _lib()
    out = C.c_double(-1.0)
    rc = lib.lp_power_norm_static(10, 600_000, None, None, None, None, None, None, 5, None,
                                  C.byref(out))
    assert rc == -1
    assert b"too large" in lib.lp_last_error()


def test_size_limit_is_exact_and_empty_sizes_need_no_gpu():
    # the array holds 2^20 doubles: 1024 partial sums, the result, v and w
    # (n each) and u (m), so m + 2 n = 2^20 - 1025 = 1,047,551 is the largest
    # size.  With NULL matrices a size that passes the check fails on the
    # pointer test instead ("NULL"), one past it on the size test.
    pkg, lib = _lib()
    out = C.c_double(-1.0)
    for m, n in ((1, 523_775), (47_551, 500_000), (1_047_549, 1)):
        assert m + 2 * n == 1_047_551
        rc = lib.lp_power_norm_static(m, n, None, None, None, None, None, None, 5, None,
                                      C.byref(out))
        assert rc == -1 and b"NULL" in lib.lp_last_error(), (m, n, lib.lp_last_error())
        rc = lib.lp_power_norm_static(m + 1, n, None, None, None, None, None, None, 5, None,
                                      C.byref(out))
        assert rc == -1 and b"too large" in lib.lp_last_error(), (m, n)
    # an empty dimension: the norm is 0 and no kernel runs
    for m, n in ((0, 7), (7, 0), (0, 0)):
        out.value = -1.0
        rc = lib.lp_power_norm_static(m, n, None, None, None, None, None, None, 5, None,
                                      C.byref(out))
        assert rc == 0 and out.value == 0.0


@pytest.mark.gpu
def test_static_power_norm_matches_solver_step_size_twice():
    import torch

    pkg, lib = _lib()
    lp = lpgen.general_structure(3000, 7000, 5, nnz_target=40000)
    dev = pkg.TorchDevice(0)
    prob = pkg.Problem(lp, dev)
    # without scaling the solver's step is 0.998 / ||A||_2 of A itself
    r = prob.solve(max_iter=1, eps_rel=0.0, ruiz_iters=0, pock_chambolle=0)
    eta_ref = r.eta
    A = lp.csr()
    AT = A.T.tocsr()

    def dev_csr(M):
        return (torch.tensor(M.indptr.astype(np.int32), device="cuda"),
                torch.tensor(M.indices.astype(np.int32), device="cuda"),
                torch.tensor(M.data.astype(np.float64), device="cuda"))

    a, at = dev_csr(A), dev_csr(AT)
    stream = torch.cuda.current_stream().cuda_stream
    ptr = lambda t: C.c_void_p(t.data_ptr())
    got = []
    for _ in range(2):
        out = C.c_double()
        rc = lib.lp_power_norm_static(lp.m, lp.n, ptr(a[0]), ptr(a[1]), ptr(a[2]), ptr(at[0]),
                                      ptr(at[1]), ptr(at[2]), 100, C.c_void_p(stream),
                                      C.byref(out))
        assert rc == 0, lib.lp_last_error()
        got.append(out.value)
        assert abs(0.998 / out.value - eta_ref) <= 1e-12 * eta_ref
    assert got[0] == got[1]


@pytest.mark.gpu
def test_static_power_norm_at_the_size_limit():
    # m + 2 n = 1,047,551 exactly: a diagonal-plus-one-entry matrix whose
    # 2-norm the allocating path (lp_solve's step size) also computes
    import scipy.sparse as sp
    import torch

    from lp_helpers import SimpleLP

    pkg, lib = _lib()
    m, n = 47_551, 500_000
    rng = np.random.default_rng(7)
    rows = np.arange(m)
    cols = rng.choice(n, size=m, replace=False)
    A = sp.csr_matrix((rng.uniform(0.5, 2.0, m), (rows, cols)), shape=(m, n))
    A = (A + sp.csr_matrix((np.full(m, 0.25), (rows, (cols + 1) % n)), shape=(m, n))).tocsr()
    A.sort_indices()
    lp = SimpleLP(A, np.ones(n), np.zeros(m), np.zeros(m), np.zeros(n), np.full(n, np.inf))
    prob = pkg.Problem(lp, pkg.TorchDevice(0))
    r = prob.solve(max_iter=1, eps_rel=0.0, ruiz_iters=0, pock_chambolle=0)
    AT = A.T.tocsr()

    def dev_csr(M):
        return [torch.tensor(M.indptr.astype(np.int32), device="cuda"),
                torch.tensor(M.indices.astype(np.int32), device="cuda"),
                torch.tensor(M.data.astype(np.float64), device="cuda")]

    a, at = dev_csr(A), dev_csr(AT)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    out = C.c_double()
    rc = lib.lp_power_norm_static(m, n, *[ptr(t) for t in a], *[ptr(t) for t in at], 100,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                  C.byref(out))
    assert rc == 0, lib.lp_last_error()
    assert abs(0.998 / out.value - r.eta) <= 1e-12 * r.eta
    prob.close()
