"""Pins for the oracle's presolve -> PDHG -> postsolve pipeline and its
original-LP check (CPU only).

The amplification LP fixes by construction how far the reduced LP's
relative KKT error can be from the original's (a known right-hand-side
shrink factor), and its planted optimum fixes the objective.
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import pipeline as PL
from oracle import presolve as PS


def rel_obj(p, q):
    return abs(p - q) / (1.0 + abs(q))


def test_generator_plants_an_optimum():
    lp = lpgen.amplified_postsolve()
    k = oracle.rel_kkt(lp, lp.x_star, lp.y_star)
    assert k["rel_kkt"] <= 1e-12
    # removing the fixed column multiplies every right-hand side by `shrink`
    pres = PS.presolve(lp)
    red = pres.reduced
    assert pres.counts["fixed_col"] == 1 and red.m == lp.m
    rhs_red = np.sort(np.abs(red.row_lo))
    rhs_org = np.sort(np.abs(lp.row_lo))
    assert np.allclose(rhs_red, 30.0 * rhs_org, rtol=1e-12)


def test_postsolve_amplifies_and_the_re_solve_recovers():
    lp = lpgen.amplified_postsolve(seed=43)
    first = PL.solve_original(lp, refine=0)
    assert first.reduced_kkt <= 1e-6
    # the same residuals, normalised by a 30x smaller ||bhat||
    assert first.kkt["rel_kkt"] > 3e-6
    assert first.kkt["rel_kkt"] <= 30.0 * first.reduced_kkt * (1 + 1e-9)
    ref = PL.solve_original(lp, refine=3)
    assert ref.status == oracle.pdhg.OPTIMAL
    assert 1 <= ref.refinements <= 3
    assert ref.kkt["rel_kkt"] <= 1e-6
    assert rel_obj(ref.kkt["p"], lp.p_star) <= 1e-6
    assert ref.iterations > first.iterations


def test_without_amplification_the_first_solve_stands():
    # the same LP without the shrink (factor 1): presolve leaves the norms
    # alone and the postsolved point is as good as the reduced one
    lp = lpgen.amplified_postsolve(seed=43, shrink=1.0)
    r = PL.solve_original(lp, refine=3)
    assert r.refinements == 0
    assert r.kkt["rel_kkt"] <= 1e-6
    assert rel_obj(r.kkt["p"], lp.p_star) <= 2e-6
