"""CPU oracle for the LP solver: plain, slow, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or
links anything here; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path.

Contents
--------
``pdhg``      rel-KKT of eq. (2), Ruiz + Pock-Chambolle scaling, power
              iteration, the PDHG operator, restarted reflected Halpern PDHG,
              infeasibility / unboundedness certificates.
``vertex``    brute-force vertex enumeration for tiny bounded LPs (a pin).
``presolve``  the presolve rules of Sec. 2-3 (fast explorers, parallel rows,
              opt-in primal propagation) and their postsolve.

Problems are passed as any object with the attributes ``m, n, row_ptr,
col_idx, val, c, obj_offset, row_lo, row_hi, col_lo, col_hi`` (the CSR form of
eq. (1)).

Parity status of each function is stated in its module header.
"""
from .pdhg import (  # noqa: F401
    Opts,
    Result,
    dual_cone_project,
    pdhg_operator,
    pdhg_solve,
    power_norm,
    rel_kkt,
    ruiz_pc_scaling,
)
