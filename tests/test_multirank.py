"""The N > 1 host logic of bench.py on CPU (world size 2, gloo): the job's
time is the slowest rank's, batch workloads scale weakly with each rank
solving its own seeded share (rank 0 the configuration's batch), and a
share is the same LPs whatever slice of the sequence generates them.

Single-LP workloads run replicas only (no collective on the data path);
batched and served LPs are independent problems, sharded with no collective.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import lpgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    job = bench.max_over_ranks(1.5 + rank, dist, "cpu")  # ranks' step times 1.5 s and 2.5 s
    first = bench.weak_share(rank, 4)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, job, first))


def test_two_ranks_time_and_shares():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]     # the slowest rank's time on every rank
    assert [r[2] for r in res] == [0, 4]         # rank r starts at item r * per_rank


def test_batch_shares_are_slices_of_one_sequence():
    whole = lpgen.c4_batch(5, m_hi=300)
    part = lpgen.c4_batch(3, m_hi=300, first=2)
    for a, b in zip(whole[2:], part):
        assert (a.m, a.n, a.nnz) == (b.m, b.n, b.nnz)
        np.testing.assert_array_equal(a.val, b.val)
        np.testing.assert_array_equal(a.c, b.c)


def test_single_rank_needs_no_process_group():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.weak_share(0, 512) == 0
