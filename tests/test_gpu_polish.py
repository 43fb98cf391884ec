"""Feasibility polishing and the separate gap tolerance on the grid engine
(through the C ABI) against the oracle's reading (oracle/pdhg.py:
feasibility_polish, kkt_met)."""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import pdhg as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_23951_gb300 as p

    p.load()
    return p


@pytest.fixture(scope="module")
def dev(pkg):
    return pkg.TorchDevice(0)


def gs(seed):
    return lpgen.general_structure(2000, 5000, seed, nnz_target=40_000, one_sided=0.2)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_polished_solve_matches_the_oracle(pkg, dev, use_graph):
    # eps 1e-8 with a gap tolerance of 1e-4: the oracle polishes at the
    # checks 384, 768, 1536 (failed) and 3072 (accepted), 3,715 iterations in
    # all against 8,705 without polishing; the phases run through the
    # captured graph or as direct launches
    lp = gs(8)
    ref = P.pdhg_solve(lp, P.Opts(eps_rel=1e-8, eps_gap=1e-4, polish=True))
    assert ref.polish["successes"] == 1
    prob = pkg.Problem(lp, dev)
    r = prob.solve(eps_rel=1e-8, eps_gap_rel=1e-4, polish=1, engine=1, use_graph=use_graph)
    assert r.termination == pkg.LP_OPTIMAL and r.polished == 1
    assert r.polish_attempts == ref.polish["attempts"]
    # the same checks decide; a phase's stop can move by one check period
    assert abs(r.iterations - ref.iterations) <= 2 * 64
    assert abs(r.polish_iterations - ref.polish["phase_iterations"]) <= 2 * 64
    x, y, _ = prob.solution()
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_p"] <= 1e-8 * (1 + 1e-6) and k["rel_d"] <= 1e-8 * (1 + 1e-6)
    assert k["rel_gap"] <= 1e-4
    assert abs(k["rel_p"] - r.rel_p) <= 1e-6 * r.rel_p + 1e-15
    assert abs(k["rel_d"] - r.rel_d) <= 1e-6 * r.rel_d + 1e-15
    prob.close()


def test_failed_attempts_resume_the_main_solve_exactly(pkg, dev):
    # at eps_gap = eps_rel every attempt fails on this LP; the main iterates
    # must then be bit for bit those of a solve without polishing, and the
    # phases only add iterations
    lp = gs(6)
    ref = P.pdhg_solve(lp, P.Opts(polish=True))
    assert ref.polish["attempts"] >= 1 and ref.polish["successes"] == 0
    prob = pkg.Problem(lp, dev)
    r0 = prob.solve(engine=1)
    x0, y0 = prob.iterate()
    s0 = prob.solution()
    r1 = prob.solve(engine=1, polish=1)
    x1, y1 = prob.iterate()
    s1 = prob.solution()
    assert r1.polish_attempts == ref.polish["attempts"] and r1.polished == 0
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(y1, y0)
    np.testing.assert_array_equal(s1[0], s0[0])
    np.testing.assert_array_equal(s1[1], s0[1])
    assert r1.restarts == r0.restarts
    assert r1.iterations == r0.iterations + r1.polish_iterations
    assert r1.polish_iterations > 0
    prob.close()


def test_polishing_in_mixed_precision_meets_the_test(pkg, dev):
    # the phases run the mixed SpMV like the main solve; the accepted pair
    # is checked on the original LP in FP64
    lp = gs(8)
    prob = pkg.Problem(lp, dev)
    r = prob.solve(eps_rel=1e-7, eps_gap_rel=1e-4, polish=1, engine=1,
                   precision=pkg.LP_MIXED)
    assert r.termination == pkg.LP_OPTIMAL and r.polish_attempts >= 1
    x, y, _ = prob.solution()
    k = oracle.rel_kkt(lp, x, y)
    tol = 1 + 1e-6
    assert k["rel_p"] <= 1e-7 * tol and k["rel_d"] <= 1e-7 * tol and k["rel_gap"] <= 1e-4 * tol
    prob.close()


@pytest.mark.parametrize("engine", [1, 2])
def test_separate_gap_tolerance(pkg, dev, engine):
    lp = lpgen.c1_small()
    prob = pkg.Problem(lp, dev)
    r0 = prob.solve(engine=engine)
    r1 = prob.solve(engine=engine, eps_gap_rel=1e-6)
    assert r1.iterations == r0.iterations  # 1e-6 is the default's gap bound
    r2 = prob.solve(engine=engine, eps_gap_rel=1e-3)
    assert r2.termination == pkg.LP_OPTIMAL and r2.iterations <= r0.iterations
    x, y, _ = prob.solution()
    k = oracle.rel_kkt(lp, x, y)
    tol = 1 + 1e-6  # the host recompute's rounding
    assert k["rel_p"] <= 1e-6 * tol and k["rel_d"] <= 1e-6 * tol and k["rel_gap"] <= 1e-3 * tol
    prob.close()


def test_polish_options_are_validated(pkg, dev):
    prob = pkg.Problem(lpgen.c1_small(), dev)
    with pytest.raises(pkg.LPError):
        prob.solve(engine=2, polish=1)
    with pytest.raises(pkg.LPError):
        prob.solve(polish=1, polish_fraction=0.0)
    with pytest.raises(pkg.LPError):
        prob.solve(eps_gap_rel=-1.0)
    # LP_ENGINE_AUTO picks the grid engine for a small LP when polishing
    r = prob.solve(polish=1, eps_rel=1e-8, eps_gap_rel=1e-4)
    assert r.termination == pkg.LP_OPTIMAL
    prob.close()
    with pytest.raises(pkg.LPError):
        pkg.Server(1 << 30, dev, polish=1)
    with pytest.raises(pkg.LPError):
        pkg.Server(1 << 30, dev, eps_gap_rel=1e-4)
