"""Batched solving and the continuous-batching server against the oracle.

Tolerances: rel-KKT <= 1e-6 bounds the duality gap by 1e-6 (1 + |p| + |d|),
not the objective error by 1e-6 (1 + |p*|); so FP64 runs that assert
objectives within 1e-6 relative of the planted optimum solve to
eps_rel = 1e-7.  Mixed precision (FP32 SpMV) solves to 1e-6 and is checked
against the FP64 optimum at 1e-5.
"""
import time

import numpy as np
import pytest

import lpgen
import oracle
from oracle import presolve as PS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_23951_gb300 as p

    p.load()
    return p


@pytest.fixture(scope="module")
def dev(pkg):
    return pkg.TorchDevice(0)


def rel_obj(p, q):
    return abs(p - q) / (1.0 + abs(q))


def small_batch(count, seed=77, m_lo=30, m_hi=600):
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=count)).astype(int)
    return [lpgen.equality_nonneg(int(m), 2 * int(m), seed + 1000 * (j + 1), 4, 30)
            for j, m in enumerate(ms)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle(pkg, dev, precision):
    lps = small_batch(24)
    eps = 1e-7 if precision == 0 else 1e-6
    srv = pkg.Server(1 << 30, dev, precision=precision, eps_rel=eps)
    probs = [pkg.Problem(lp, dev) for lp in lps]
    tickets = [srv.submit(p) for p in probs]
    res = srv.run_all(tickets)
    tol = 1e-6 if precision == 0 else 1e-5
    for lp, t in zip(lps, tickets):
        r, x, y = res[t]
        assert r.termination == pkg.LP_OPTIMAL, r.as_dict()
        assert r.rel_kkt <= eps
        k = oracle.rel_kkt(lp, x, y)
        assert k["rel_kkt"] <= 2 * eps, k
        assert rel_obj(r.primal_obj, lp.p_star) <= tol
    st = srv.stats()
    assert st["finished"] == len(lps) and st["queued"] == 0
    srv.close()


def test_single_lp_batch_of_one_matches_single_path(pkg, dev):
    lp = lpgen.c1_small()
    ref = oracle.pdhg_solve(lp)
    srv = pkg.Server(1 << 28, dev, precision=0)
    p = pkg.Problem(lp, dev)
    t = srv.submit(p)
    r, x, y = srv.run_all([t])[t]
    assert r.termination == pkg.LP_OPTIMAL and r.rel_kkt <= 1e-6
    assert rel_obj(r.primal_obj, ref.kkt["p"]) <= 1e-6
    # same algorithm, same arithmetic type: the iteration count matches the
    # oracle's unless a restart test lands on a near-tie
    assert abs(r.iterations - ref.iterations) <= 128
    srv.close()


@pytest.mark.parametrize("precision,eps,tol", [(0, 1e-7, 1e-6), (1, 1e-6, 1e-5)])
def test_alone_and_in_the_mix_agree(pkg, dev, precision, eps, tol):
    target = lpgen.equality_nonneg(300, 600, 4242, 4, 30)
    others = small_batch(30, seed=99)
    srv = pkg.Server(1 << 30, dev, precision=precision, eps_rel=eps)
    pa = pkg.Problem(target, dev)
    ta = srv.submit(pa)
    ra, xa, ya = srv.run_all([ta])[ta]
    srv.close()
    srv = pkg.Server(1 << 30, dev, precision=precision, eps_rel=eps)
    probs = [pkg.Problem(lp, dev) for lp in others[:15]]
    tickets = [srv.submit(p) for p in probs]
    pb = pkg.Problem(target, dev)
    tb = srv.submit(pb)
    probs2 = [pkg.Problem(lp, dev) for lp in others[15:]]
    tickets += [srv.submit(p) for p in probs2]
    res = srv.run_all(tickets + [tb])
    rb, xb, yb = res[tb]
    assert ra.termination == rb.termination == pkg.LP_OPTIMAL
    assert rel_obj(ra.primal_obj, rb.primal_obj) <= tol
    assert rel_obj(ra.primal_obj, target.p_star) <= tol
    assert ra.rel_kkt <= eps and rb.rel_kkt <= eps
    srv.close()


def test_cancel_and_budget(pkg, dev):
    srv = pkg.Server(1 << 26, dev, precision=1)
    lp = lpgen.equality_nonneg(200, 400, 5, 4, 30)
    t = srv.submit(pkg.Problem(lp, dev))
    srv.cancel(t)
    r, _, _ = srv.run_all([t])[t]
    assert r.termination == 6  # LP_CANCELLED
    big = lpgen.equality_nonneg(60000, 120000, 6, 20, 30)
    with pytest.raises(pkg.LPError) as ei:
        srv.submit(pkg.Problem(big, dev))
    assert ei.value.code == -5
    srv.close()


def test_worker_thread_continuous_batching(pkg, dev):
    lps = small_batch(20, seed=5)
    srv = pkg.Server(1 << 30, dev, worker=True, precision=1)
    probs = [pkg.Problem(lp, dev) for lp in lps]
    first = [srv.submit(p) for p in probs[:10]]
    time.sleep(0.05)  # the first wave is running when the second arrives
    second = [srv.submit(p) for p in probs[10:]]
    pending = set(first + second)
    out = {}
    t0 = time.time()
    while pending and time.time() - t0 < 120:
        for t in list(pending):
            got = srv.poll(t)
            if got is not None:
                out[t] = got
                pending.discard(t)
        time.sleep(0.002)
    assert not pending
    for lp, t in zip(lps, first + second):
        r, x, y = out[t]
        assert r.termination == pkg.LP_OPTIMAL
        assert rel_obj(r.primal_obj, lp.p_star) <= 1e-5
    srv.close()


def test_presolved_requests_postsolve_to_kkt(pkg, dev):
    lps = [lpgen.general_structure(400 + 50 * j, 1000 + 120 * j, 300 + j, nnz_target=6000)
           for j in range(4)]
    srv = pkg.Server(1 << 30, dev, precision=0, eps_rel=1e-7)
    probs = [pkg.Problem(lp, dev) for lp in lps]
    for p in probs:
        p.presolve()
    tickets = [srv.submit(p) for p in probs]
    res = srv.run_all(tickets)
    for lp, p, t in zip(lps, probs, tickets):
        r, _, _ = res[t]
        assert r.termination == pkg.LP_OPTIMAL
        x, y, z = p.postsolve()
        k = oracle.rel_kkt(lp, x, y)
        assert r.rel_kkt_original <= 1e-7
        assert k["rel_kkt"] <= 1e-7 * (1 + 1e-6)
        assert rel_obj(k["p"], lp.p_star) <= 1e-6
    srv.close()


def test_large_request_runs_on_the_solo_lane_beside_batched_ones(pkg, dev):
    # at or above the solo size the server solves a request with the
    # single-LP grid path on its own stream while the small ones keep batching
    solo = 400_000
    big = lpgen.general_structure(24_000, 60_000, 17, nnz_target=600_000)
    smalls = small_batch(8, seed=8)
    srv = pkg.Server(8 << 30, dev, worker=True, precision=0)
    srv.tune(solo_nnz=solo)
    pb = pkg.Problem(big, dev)
    pb.presolve()
    assert pb.dims()[2] >= solo, "presolved request below the solo size"
    probs = [pkg.Problem(lp, dev) for lp in smalls]
    tb = srv.submit(pb)
    ts = [srv.submit(p) for p in probs]
    pending = set([tb] + ts)
    out = {}
    t0 = time.time()
    while pending and time.time() - t0 < 300:
        for t in list(pending):
            got = srv.poll(t)
            if got is not None:
                out[t] = got
                pending.discard(t)
        time.sleep(0.005)
    assert not pending
    r, _, _ = out[tb]
    assert r.termination == pkg.LP_OPTIMAL and r.rel_kkt <= 1e-6
    x, y, _ = pb.postsolve()
    k = oracle.rel_kkt(big, x, y)
    assert r.rel_kkt_original <= 1e-6 and k["rel_kkt"] <= 1e-6 * (1 + 1e-6)
    for lp, t in zip(smalls, ts):
        r, _, _ = out[t]
        assert r.termination == pkg.LP_OPTIMAL
        assert rel_obj(r.primal_obj, lp.p_star) <= 1e-5
    srv.close()


@pytest.mark.parametrize("lane", ["batched", "solo"])
def test_served_request_is_re_solved_when_postsolve_amplifies(pkg, dev, lane):
    # the amplified LP through the server: the poll that finds the postsolved
    # point off on the original LP queues a warm-started re-solve at 1e-7 and
    # the ticket stays pending until it is done
    lp = lpgen.amplified_postsolve(seed=43)
    srv = pkg.Server(1 << 30, dev, worker=True, precision=0)
    if lane == "solo":
        srv.tune(solo_nnz=1000)
    p = pkg.Problem(lp, dev)
    p.presolve()
    t = srv.submit(p)
    got = None
    t0 = time.time()
    while got is None and time.time() - t0 < 120:
        got = srv.poll(t)
        time.sleep(0.002)
    assert got is not None
    r = got[0]
    assert r.termination == pkg.LP_OPTIMAL and r.refinements >= 1
    x, y, _ = p.postsolve()
    k = oracle.rel_kkt(lp, x, y)
    assert r.rel_kkt_original <= 1e-6 and k["rel_kkt"] <= 1e-6 * (1 + 1e-6)
    assert abs(k["rel_kkt"] - r.rel_kkt_original) <= 1e-6 * r.rel_kkt_original
    assert rel_obj(k["p"], lp.p_star) <= 1e-6
    srv.close()


def test_batch_iterates_match_oracle_elementwise(pkg, dev):
    # 20 LPs from 30 to 20,000 rows (three size buckets) run together, with
    # the step size and weight fixed: after 50 and 130 iterations each
    # returned point T(z) matches the oracle's entry by entry.  A 10 us launch
    # budget gives every slot one block of K iterations per launch, so a
    # slot's iterations run across several launches and the autotuner's
    # cluster x CTA shapes (it tries one per launch while tuning).
    # The same with every bucket launch replayed from a CUDA graph and issued
    # directly: while the autotuner is still trying shapes (three launches
    # per slot here) the shape sequence is fixed, so the two agree bit for bit.
    ms = np.exp(np.linspace(np.log(30), np.log(20000), 20)).astype(int)
    lps = [lpgen.equality_nonneg(int(m), 2 * int(m), 5100 + j, 4, 30) for j, m in enumerate(ms)]
    eta, om = 0.05, 1.3
    for iters in (50, 130):
        got = {}
        for use_graph in (1, 0):
            pkg.tile_cache_clear()  # the same tile shapes for the slots of both runs
            srv = pkg.Server(1 << 31, dev, precision=0, max_iter=iters, eps_rel=0.0,
                             step_size=eta, primal_weight=om, use_graph=use_graph)
            srv.tune(launch_ms=0.01)
            probs = [pkg.Problem(lp, dev) for lp in lps]
            tickets = [srv.submit(p) for p in probs]
            res = srv.run_all(tickets)
            st = srv.stats()
            gs = srv.graph_stats()
            # three buckets, each slot over at least ceil(iters / 64) launches
            assert st["launches"] >= 3 * ((iters + 63) // 64)
            if use_graph:
                assert gs["graph_launches"] == st["periods"] and 3 <= gs["graphs"] <= 3 * 6
            else:
                assert gs["graph_launches"] == 0 and gs["graphs"] == 0
            got[use_graph] = [res[t] for t in tickets]
            for lp, (r, x, y) in zip(lps, got[use_graph]):
                ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=iters, eps_rel=0.0), eta=eta,
                                        omega0=om)
                assert r.termination == pkg.LP_ITER_LIMIT and r.iterations == iters
                assert r.restarts == ref.restarts
                ex = np.max(np.abs(x - ref.x)) / max(1.0, np.max(np.abs(ref.x)))
                ey = np.max(np.abs(y - ref.y)) / max(1.0, np.max(np.abs(ref.y)))
                assert ex <= 1e-10 and ey <= 1e-10, (lp.m, iters, ex, ey)
            srv.close()
        for (r1, x1, y1), (r0, x0, y0) in zip(got[1], got[0]):
            np.testing.assert_array_equal(x1, x0)
            np.testing.assert_array_equal(y1, y0)


def test_batch_tile_tuner_keeps_the_fastest_shape(pkg, dev):
    # two request classes of 20 LPs (m 300 and 3,000; 10-14 entries per row):
    # all 40 are packed while their class is still trying, so each class's
    # six tile shapes get three or four samples; then every class keeps the
    # shape with the least mean device time per nonzero-iteration, which
    # the next batch's requests get.  Every request solves to 1e-6 whatever
    # its shape.
    import math

    pkg.tile_cache_clear()
    lps = ([lpgen.equality_nonneg(300, 600, 7100 + j, 10, 14) for j in range(20)]
           + [lpgen.equality_nonneg(3000, 6000, 7200 + j, 10, 14) for j in range(20)])
    srv = pkg.Server(1 << 31, dev, precision=0)
    probs = [pkg.Problem(lp, dev) for lp in lps]
    tickets = [srv.submit(p) for p in probs]
    res = srv.run_all(tickets)
    for lp, t in zip(lps, tickets):
        r, x, y = res[t]
        assert r.termination == pkg.LP_OPTIMAL and r.rel_kkt <= 1e-6
        assert oracle.rel_kkt(lp, x, y)["rel_kkt"] <= 1e-6 * (1 + 1e-6)
    keys = {(int(math.floor(math.log2(lp.m) / 2)), int(math.floor(math.log2(lp.nnz / lp.m))))
            for lp in lps}
    tt = {(c["m_bucket"], c["len_bucket"]): c for c in srv.tile_tuning()}
    assert keys <= set(tt)
    assert len(keys) == 2
    for k in keys:
        c = tt[k]
        assert min(c["samples"]) >= 2 and c["chosen"] >= 0
        assert c["mean_ns"][c["chosen"]] == min(c["mean_ns"])
    # the next batch packs each class under its chosen shape (no new samples)
    before = {k: sum(tt[k]["samples"]) for k in keys}
    res2 = srv.run_all([srv.submit(pkg.Problem(lp, dev)) for lp in lps[:4] + lps[-4:]])
    assert all(r.termination == pkg.LP_OPTIMAL for r, _, _ in res2.values())
    tt2 = {(c["m_bucket"], c["len_bucket"]): c for c in srv.tile_tuning()}
    for k in keys:
        if tt[k]["chosen"] >= 0:
            assert sum(tt2[k]["samples"]) == before[k] and tt2[k]["chosen"] == tt[k]["chosen"]
    srv.close()
