"""Host helpers of bench.py (CPU): the termination histogram, the option
plumbing into lp_solve_opts / the presolve mask, and the FIFO latency of the
single-request comparator."""
import types

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b

    return b


def test_termination_histogram(bench):
    assert bench.term_hist([0, 0, 4, 1, 0]) == {"0": 3, "4": 1, "1": 1}
    assert bench.term_hist([]) == {}


def test_solver_options_and_presolve_mask(bench):
    args = types.SimpleNamespace(infeas_every=-1, propagation=False)
    assert bench.solver_kw(args) == {}
    args.infeas_every = 0
    assert bench.solver_kw(args) == {"infeas_every": 0}
    pkg = types.SimpleNamespace(LP_RULE_ALL=1023, LP_RULE_PRIMAL_PROPAGATION=1024)
    assert bench.presolve_rules(pkg, args) == 1023
    args.propagation = True
    assert bench.presolve_rules(pkg, args) == 2047


def test_kernel_hash_is_stable(bench):
    h = bench.kernel_source_hash()
    assert isinstance(h, str) and len(h) == 16 and h == bench.kernel_source_hash()


def test_fifo_latencies(bench):
    # idle server: latency = service time; a burst queues behind earlier work
    assert bench.fifo_latencies([0.0, 10.0], [1.0, 2.0]) == [1.0, 2.0]
    assert bench.fifo_latencies([0.0, 0.5, 0.6], [1.0, 1.0, 1.0]) == [1.0, 1.5, 2.4]


def test_iteration_bytes_follow_the_per_iteration_formula():
    # FP64: B = 2 nnz (8 + 4) + 4 (m + n) + 8 (8 n + 6 m), plus the two
    # trailing row offsets; the mixed SpMV halves the values and K2 also
    # writes y as a float pair
    import bench

    m, n, nnz = 1000, 2500, 30000
    assert bench.iter_bytes(m, n, nnz, False) == 2 * nnz * 12 + 4 * (m + n) + 8 * (8 * n + 6 * m) + 8
    b32 = bench.iter_bytes(m, n, nnz, True)
    assert b32 == 2 * nnz * 8 + 4 * (m + n) + 8 + 8 * m + 48 * n + 8 * n + 8 * n + 40 * m + 8 * m
