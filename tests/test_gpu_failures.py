"""Failure paths, all made on the host: an allocator that refuses, an LP the
presolve proves infeasible, a request cancelled while it runs, and the
per-check trace.  Also: the batch kernel's exact iteration-limit semantics
against the single-LP engine."""
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import lpgen
from lp_helpers import SimpleLP

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_23951_gb300 as p

    p.load()
    return p


@pytest.fixture(scope="module")
def dev(pkg):
    return pkg.TorchDevice(0)


class RefusingDevice:
    """Device context whose allocator always returns NULL."""

    def __init__(self, capi, stream):
        self._alloc = capi.ALLOC_FN(lambda nbytes, user: None)
        self._free = capi.FREE_FN(lambda ptr, user: None)
        self.ctx = capi.lp_device_ctx(self._alloc, self._free, None,
                                      capi.C.c_void_p(stream.cuda_stream), 0)


@pytest.mark.parametrize("engine", [1, 2])
def test_refusing_allocator_is_oom(pkg, dev, engine):
    from paper_2604_23951_gb300 import capi

    bad = RefusingDevice(capi, dev.stream)
    prob = pkg.Problem(lpgen.c1_small(), bad)
    with pytest.raises(pkg.LPError) as ei:
        prob.solve(engine=engine)
    assert ei.value.code == -2  # LP_ERR_OOM
    prob.close()
    with pytest.raises(pkg.LPError) as ei:
        pkg.Server(1 << 26, bad)
    assert ei.value.code == -2


def test_presolve_infeasible_is_reported(pkg, dev):
    # x >= 1 and the singleton row x <= 0
    lp = SimpleLP([[1.0, 1.0], [1.0, 0.0]], [1.0, 1.0], [-np.inf, -np.inf], [5.0, 0.0],
                  [1.0, 0.0], [np.inf, np.inf])
    prob = pkg.Problem(lp, dev)
    info = prob.presolve()
    assert info.status == 1  # LP_PRESOLVE_INFEASIBLE
    r = prob.solve()
    assert r.termination == pkg.LP_INFEASIBLE


def test_cancel_while_running(pkg, dev):
    lp = lpgen.equality_nonneg(4000, 8000, 31, 4, 30)
    srv = pkg.Server(1 << 30, dev, worker=True, precision=0, eps_rel=1e-12, max_iter=5_000_000)
    t = srv.submit(pkg.Problem(lp, dev))
    t0 = time.time()
    while srv.stats()["admitted"] < 1 and time.time() - t0 < 30:
        time.sleep(0.01)
    time.sleep(0.2)  # it is iterating on the device now
    srv.cancel(t)
    got = None
    while got is None and time.time() - t0 < 60:
        got = srv.poll(t)
        time.sleep(0.01)
    assert got is not None
    assert got[0].termination == 6  # LP_CANCELLED
    srv.close()


@pytest.mark.parametrize("iters", [64, 130])
def test_batch_iteration_limit_matches_single_engine(pkg, dev, iters):
    # the batch kernel stops inside a block of K iterations exactly like the
    # grid engine and returns the same last T(z)
    lp = lpgen.general_structure(700, 1800, 41, nnz_target=12000, one_sided=0.2)
    eta, om = 0.05, 0.9
    p1 = pkg.Problem(lp, dev)
    r1 = p1.solve(max_iter=iters, eps_rel=0.0, step_size=eta, primal_weight=om, engine=1)
    x1, y1, _ = p1.solution()
    srv = pkg.Server(1 << 28, dev, precision=0, max_iter=iters, eps_rel=0.0, step_size=eta,
                     primal_weight=om)
    p2 = pkg.Problem(lp, dev)
    t = srv.submit(p2)
    r2, x2, y2 = srv.run_all([t])[t]
    srv.close()
    assert r1.termination == r2.termination == pkg.LP_ITER_LIMIT
    assert r1.iterations == r2.iterations == iters
    scale = max(1.0, np.max(np.abs(x1)))
    assert np.max(np.abs(x1 - x2)) / scale <= 1e-9
    assert np.max(np.abs(y1 - y2)) / max(1.0, np.max(np.abs(y1))) <= 1e-9
    assert abs(r1.rel_kkt - r2.rel_kkt) <= 1e-8 * (1 + r1.rel_kkt)


def test_trace_writes_one_json_line_per_readback(tmp_path):
    path = tmp_path / "trace.jsonl"
    code = ("import sys; sys.path.insert(0, %r); import lpgen, paper_2604_23951_gb300 as p; "
            "p.load(); d = p.TorchDevice(0); q = p.Problem(lpgen.c1_small(), d); "
            "r = q.solve(engine=1); print(r.iterations)" % ROOT)
    env = dict(os.environ, LP_TRACE=str(path))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    iters = int(out.stdout.strip().splitlines()[-1])
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert lines and all(l["engine"] == "grid" for l in lines)
    assert lines[-1]["rel_kkt"] <= 1e-6
    assert max(l["t"] for l in lines) <= iters + 64


def test_server_answers_presolve_infeasible_at_once(pkg, dev):
    lp = SimpleLP([[1.0, 1.0], [1.0, 0.0]], [1.0, 1.0], [-np.inf, -np.inf], [5.0, 0.0],
                  [1.0, 0.0], [np.inf, np.inf])
    prob = pkg.Problem(lp, dev)
    prob.presolve()
    srv = pkg.Server(1 << 26, dev)
    t = srv.submit(prob)
    got = srv.poll(t)  # no pump needed: decided at submission
    assert got is not None and got[0].termination == pkg.LP_INFEASIBLE
    srv.close()


@pytest.mark.parametrize("bad", [{"infeas_every": -1}, {"eps_infeas": -1.0},
                                 {"primal_weight_clamp": 0.5}, {"primal_weight_clamp": -2.0}])
def test_invalid_solver_options_are_rejected(pkg, dev, bad):
    prob = pkg.Problem(lpgen.c1_small(), dev)
    with pytest.raises(pkg.LPError) as ei:
        prob.solve(**bad)
    assert ei.value.code == -1  # LP_ERR_INVALID, before any device work
    prob.close()
