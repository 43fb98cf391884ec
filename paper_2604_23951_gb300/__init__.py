"""GB300-native restarted-PDHG LP solver with host presolve/postsolve.

The compute path is the native library built from ``csrc/`` (CUDA for
sm_103a + host C++), reached through the C ABI of ``include/lp.h``.  This
package only marshals arguments (``capi``); PyTorch supplies device memory
and streams.
"""
from .capi import (  # noqa: F401
    LP_FP64,
    LP_MIXED,
    LP_ENGINE_AUTO,
    LP_ENGINE_GRID,
    LP_ENGINE_CLUSTER,
    LP_RULE_ALL,
    LP_RULE_EMPTY_ROW,
    LP_RULE_EMPTY_COL,
    LP_RULE_FIXED_COL,
    LP_RULE_SINGLETON_ROW,
    LP_RULE_REDUNDANT_ROW,
    LP_RULE_DOUBLETON,
    LP_RULE_FREE_COL_SINGLETON,
    LP_RULE_COL_SINGLETON_INEQ,
    LP_RULE_PARALLEL_ROWS,
    LP_RULE_DUAL_PROPAGATION,
    LP_RULE_PARALLEL_COLS,
    LP_RULE_PRIMAL_PROPAGATION,
    LP_RULE_VARIABLE_LOCKS,
    LP_OPTIMAL,
    LP_ITER_LIMIT,
    LP_TIME_LIMIT,
    LP_NUMERICAL,
    LP_INFEASIBLE,
    LP_UNBOUNDED,
    LP_CANCELLED,
    LPError,
    Problem,
    Server,
    TorchDevice,
    load,
    plan_rows,
    plan_rows_shape,
    tile_cache_clear,
    solve_opts,
)
