"""Infeasibility / unboundedness detection on the GPU (both engines and the
batch server) against the oracle's statuses on the same LPs; feasible LPs
are never flagged (every other GPU test solves feasible LPs to optimality
with the test on)."""
import numpy as np
import pytest

import oracle
from infeasible_lps import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_23951_gb300 as p

    p.load()
    return p


@pytest.fixture(scope="module")
def dev(pkg):
    return pkg.TorchDevice(0)


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("name,make,status", CASES)
def test_detection_matches_oracle(pkg, dev, engine, name, make, status):
    lp = make()
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=20000))
    assert ref.status == status
    prob = pkg.Problem(lp, dev)
    r = prob.solve(max_iter=20000, engine=engine)
    assert r.termination == status, (name, r.termination, r.iterations)
    # detection happens at a test check (every 4th check of 64 iterations)
    assert (r.iterations - 1) % 256 == 0
    assert r.iterations <= 4 * ref.iterations + 256


@pytest.mark.parametrize("engine", [1, 2])
def test_detection_off_runs_to_the_limit(pkg, dev, engine):
    lp = CASES[0][1]()
    r = pkg.Problem(lp, dev).solve(max_iter=1000, infeas_every=0, engine=engine)
    assert r.termination == pkg.LP_ITER_LIMIT


def test_server_reports_each_status(pkg, dev):
    import lpgen

    srv = pkg.Server(1 << 28, dev, precision=0)
    probs = [pkg.Problem(make(), dev) for _, make, _ in CASES]
    probs.append(pkg.Problem(lpgen.c1_small(), dev))
    want = [s for _, _, s in CASES] + [pkg.LP_OPTIMAL]
    tickets = [srv.submit(p) for p in probs]
    res = srv.run_all(tickets)
    got = [res[t][0].termination for t in tickets]
    srv.close()
    assert got == want
