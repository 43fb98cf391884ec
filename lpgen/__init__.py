"""Seeded synthetic planted LP generators.

This package only builds problem instances; it holds none of the solver's
arithmetic (no scaling, no PDHG step, no presolve rule).  Both the CUDA path
and the CPU oracle consume what it produces, and neither depends on the other.

Every instance is a planted LP

    minimize c^T x  s.t.  row_lo <= A x <= row_hi,  col_lo <= x <= col_hi

(the problem form of eq. (1)) whose optimum is fixed by construction: a primal
point x*, a dual point (y*, z*) are drawn first, the bounds are placed so that
complementary slackness (the sign conditions of eq. (2)) holds, and
c = A^T y* + z*.  Hence p* = c^T x* equals the dual objective at (y*, z*).
"""
from .planted import (  # noqa: F401
    BASE_SEED,
    PlantedLP,
    amplified_postsolve,
    c1_small,
    c2_presolvable,
    c3_powerlaw,
    c4_batch,
    c5_stream,
    general_structure,
    medium_structure,
    equality_nonneg,
    tiny_box,
)
