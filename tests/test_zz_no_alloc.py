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
