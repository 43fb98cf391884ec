"""Oracle of the whole path for one LP: presolve, PDHG on the reduced LP,
postsolve, and the check of the result on the original LP.

TEST INFRASTRUCTURE ONLY (see the package header).  FP64.

READING (the paper states that presolve returns an approximate solution of
the original LP, Sec. 2.1 and Sec. 3.3, without a rule for when that
approximation is not good enough): the reduced LP is solved to eps_rel; the
postsolved point's relative KKT error (eq. (2), the measure of
``pdhg.rel_kkt``) is then measured on the ORIGINAL LP, and while it fails the
stopping test (``pdhg.kkt_met``: rel-KKT <= eps_rel unless a separate gap
tolerance is set) the reduced LP is solved again with tolerances ten times tighter,
warm-started from the previous solution, at most ``refine`` times.  The
reduction can amplify the error because the relative measure normalises by
the problem's own ||bhat|| and ||c||, which presolve changes (a fixed column
moves right-hand sides), while the residuals themselves carry over.

Pins (tests/test_oracle_pipeline.py): on ``lpgen.amplified_postsolve`` (a
fixed column that shrinks every right-hand side by a known factor) the first
postsolved point misses eps_rel on the original LP by up to that factor, the
refined one meets it, and its objective is the planted optimum; on LPs
without that structure no re-solve happens.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import pdhg as P
from . import presolve as PS


@dataclass
class PipelineResult:
    status: int
    x: np.ndarray  # original LP
    y: np.ndarray
    z: np.ndarray
    kkt: dict  # rel_kkt of (x, y) on the original LP
    refinements: int
    iterations: int
    reduced_kkt: float  # rel-KKT of the last reduced solve


def solve_original(lp, opts: P.Opts | None = None, refine: int = 3) -> PipelineResult:
    opts = opts or P.Opts()
    pres = PS.presolve(lp)
    red = pres.reduced
    if pres.status not in (PS.REDUCED, PS.SOLVED):
        return PipelineResult(status={PS.INFEASIBLE: P.INFEASIBLE}.get(pres.status, P.UNBOUNDED),
                              x=np.zeros(lp.n), y=np.zeros(lp.m), z=np.zeros(lp.n), kkt={},
                              refinements=0, iterations=0, reduced_kkt=float("nan"))
    eps = opts.eps_rel
    r = P.pdhg_solve(red, opts)
    iters = r.iterations
    refinements = 0
    while True:
        x, y, z = PS.postsolve(pres, r.x, r.y, r.z)
        k = P.rel_kkt(lp, x, y)
        if P.kkt_met(k, opts) or refinements == refine or r.status != P.OPTIMAL:
            break
        eps *= 0.1
        gap = None if opts.eps_gap is None else opts.eps_gap * 0.1 ** (refinements + 1)
        o2 = P.Opts(**{**opts.__dict__, "eps_rel": eps, "eps_gap": gap})
        r = P.pdhg_solve(red, o2, x_init=r.x, y_init=r.y)
        iters += r.iterations
        refinements += 1
    return PipelineResult(status=r.status, x=x, y=y, z=z, kkt=k, refinements=refinements,
                          iterations=iters, reduced_kkt=r.kkt["rel_kkt"])
