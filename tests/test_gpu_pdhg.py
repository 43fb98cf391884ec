"""GPU PDHG (through the C ABI) against the CPU oracle.

Tolerances: iterates 1e-10 relative to max(1, ||oracle||_inf) (FP64, step and
weight passed explicitly); final objectives 1e-6 relative; both sides reach
rel-KKT <= 1e-6.
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import pipeline as oracle_pipeline
from oracle import presolve as PS
from lp_helpers import SimpleLP

pytestmark = pytest.mark.gpu

INF = np.inf


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_23951_gb300 as p

    p.load()
    return p


@pytest.fixture(scope="module")
def dev(pkg):
    return pkg.TorchDevice(0)


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))) if b.size else 0.0


def rel_obj(p, q):
    return abs(p - q) / (1.0 + abs(q))


ENGINES = [1, 2]  # LP_ENGINE_GRID, LP_ENGINE_CLUSTER


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("iters", [1, 2, 5, 17, 50, 64, 65, 130])
def test_first_iterates_match_oracle_c1(pkg, dev, iters, engine):
    lp = lpgen.c1_small()
    eta, om = 0.05, 1.3
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=iters, eps_rel=0.0), eta=eta, omega0=om)
    prob = pkg.Problem(lp, dev)
    r = prob.solve(max_iter=iters, eps_rel=0.0, step_size=eta, primal_weight=om, engine=engine)
    assert r.termination == pkg.LP_ITER_LIMIT and r.iterations == iters
    xi, yi = prob.iterate()
    assert relerr(xi, ref.x_iter) <= 1e-10
    assert relerr(yi, ref.y_iter) <= 1e-10
    # the returned point is the last T(z) evaluated, as in the oracle
    x, y, _ = prob.solution()
    assert relerr(x, ref.x) <= 1e-10 and relerr(y, ref.y) <= 1e-10
    assert abs(r.rel_kkt - ref.kkt["rel_kkt"]) <= 1e-9 * (1 + ref.kkt["rel_kkt"])


def test_iterates_powerlaw_all_row_classes(pkg, dev):
    # row lengths from 1 to thousands: every lanes-per-row class and the
    # block-per-row class are exercised, with a ragged last tile in each
    lp = lpgen.c3_powerlaw(seed=7, m=3000, n=8000, row_nnz_target=60000, n_dense=20,
                           dense_len=2500, kmax=6000)
    eta, om = 0.02, 0.7
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=40, eps_rel=0.0), eta=eta, omega0=om)
    for engine in ENGINES:
        prob = pkg.Problem(lp, dev)
        prob.solve(max_iter=40, eps_rel=0.0, step_size=eta, primal_weight=om, engine=engine)
        xi, yi = prob.iterate()
        assert relerr(xi, ref.x_iter) <= 1e-10
        assert relerr(yi, ref.y_iter) <= 1e-10
        prob.close()


@pytest.mark.parametrize("engine", ENGINES)
def test_step_size_and_weight_match_oracle(pkg, dev, engine):
    lp = lpgen.general_structure(500, 1200, 3, nnz_target=7000, one_sided=0.2)
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=1, eps_rel=0.0))
    prob = pkg.Problem(lp, dev)
    r = prob.solve(max_iter=1, eps_rel=0.0, engine=engine)
    assert abs(r.eta - ref.eta) <= 1e-12 * ref.eta
    assert abs(r.omega - ref.omega0) <= 1e-12 * ref.omega0


@pytest.mark.parametrize("engine", ENGINES)
def test_c1_solves_to_tolerance(pkg, dev, engine):
    lp = lpgen.c1_small()
    ref = oracle.pdhg_solve(lp)
    prob = pkg.Problem(lp, dev)
    r = prob.solve(engine=engine)
    assert r.termination == pkg.LP_OPTIMAL
    assert r.rel_kkt <= 1e-6
    x, y, z = prob.solution()
    k = oracle.rel_kkt(lp, x, y)
    assert k["rel_kkt"] <= 1e-6
    assert rel_obj(r.primal_obj, ref.kkt["p"]) <= 1e-6
    assert rel_obj(r.primal_obj, lp.p_star) <= 1e-6
    # the restart schedule agrees until the trajectories split on a threshold
    assert r.restarts >= 1


@pytest.mark.parametrize("graph", [0, 1])
def test_graph_and_direct_launches_agree_bitwise(pkg, dev, graph):
    lp = lpgen.general_structure(400, 1000, 8, nnz_target=6000)
    prob = pkg.Problem(lp, dev)
    r1 = prob.solve(max_iter=300, eps_rel=0.0, use_graph=1, engine=1)
    x1, y1 = prob.iterate()
    r2 = prob.solve(max_iter=300, eps_rel=0.0, use_graph=graph, engine=1)
    x2, y2 = prob.iterate()
    assert r1.restarts == r2.restarts
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(y1, y2)


@pytest.mark.parametrize("engine", ENGINES)
def test_presolve_solve_postsolve_is_kkt(pkg, dev, engine):
    lp = lpgen.general_structure(1500, 3800, 12, nnz_target=30000, one_sided=0.1)
    prob = pkg.Problem(lp, dev)
    info = prob.presolve()
    assert info.m < lp.m
    r = prob.solve(engine=engine)
    assert r.termination == pkg.LP_OPTIMAL and r.rel_kkt <= 1e-6
    x, y, z = prob.postsolve()
    k = oracle.rel_kkt(lp, x, y)
    # the original-LP check holds the postsolved point to eps_rel = 1e-6
    assert r.rel_kkt_original <= 1e-6
    assert k["rel_kkt"] <= 1e-6 * (1 + 1e-6)
    assert abs(k["rel_kkt"] - r.rel_kkt_original) <= 1e-6 * r.rel_kkt_original
    assert rel_obj(k["p"], lp.p_star) <= 1e-6
    # the oracle on the same reduced problem reaches the same objective
    ref = oracle.pdhg_solve(PS.presolve(lp).reduced)
    assert rel_obj(r.primal_obj, ref.kkt["p"]) <= 1e-6


@pytest.mark.parametrize("engine", ENGINES)
def test_mixed_precision_reaches_tolerance(pkg, dev, engine):
    lp = lpgen.c1_small()
    prob = pkg.Problem(lp, dev)
    r = prob.solve(precision=pkg.LP_MIXED, engine=engine)
    assert r.termination == pkg.LP_OPTIMAL and r.rel_kkt <= 1e-6
    assert rel_obj(r.primal_obj, lp.p_star) <= 1e-5


def _one_mixed_iteration(pkg, dev, lp, engine, eta, om, scaled, y_init=None):
    prob = pkg.Problem(lp, dev)
    r = prob.solve(max_iter=1, eps_rel=0.0, step_size=eta, primal_weight=om, engine=engine,
                   precision=pkg.LP_MIXED, y_init=y_init, ruiz_iters=10 if scaled else 0,
                   pock_chambolle=int(scaled))
    assert r.iterations == 1 and r.fp32_iterations == 1
    xi, yi = prob.iterate()
    prob.close()
    return xi, yi


@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("engine", ENGINES)
def test_mixed_spmv_error_is_the_matrix_rounding_only(pkg, dev, engine, scaled):
    # One iteration of the mixed mode against the FP64 oracle on rows of
    # 3,000 positive terms.  The mixed SpMV multiplies FP32 matrix values by
    # the gathered vector held as a float pair and accumulates with Dot2, so
    # row i of its result differs from the exact one by the matrix rounding
    # (at most u (|A~| |v|)_i, u = 2^-24) plus the error of the side sums,
    # about (entries per lane) u^2 (each lane adds at most 32 entries before
    # the exact TwoSum combination).  Unscaled, the small-integer matrix is
    # exact in float and the result must agree to 2^-38 of (|A~| |v|)_i: a
    # float-rounded vector would be off by about 2^-31.6 of it on these rows
    # (u / 2 per term, random signs) and a plain FP32 running sum by far more.
    # Scaled, the bound is 2.5u.
    # rho = 1, lambda_0 = 1/2 and a zero anchor make the first iterate T(z)
    # itself, and the projections are 1-Lipschitz, so the SpMV bound carries
    # over scaled by tau (x) or sigma (y).
    rel = 2.5 * 2.0 ** -24 if scaled else 2.0 ** -38
    rng = np.random.default_rng(21)
    eta, om = 0.3 if scaled else 1e-4, 1.0
    tau, sigma = eta / om, eta * om
    opts = oracle.Opts(max_iter=1, eps_rel=0.0, ruiz_iters=10 if scaled else 0,
                       pock_chambolle=scaled)
    # K2 (rows of A): 24 equality rows of 3,000 entries, x_0 = 0
    A = rng.integers(1, 4, (24, 3000)).astype(float)
    b = A @ np.ones(3000)
    lp = SimpleLP(A, -rng.uniform(0.5, 1.5, 3000), b, b, np.zeros(3000), np.full(3000, INF))
    sc = oracle.pdhg.Scaled(lp, opts)
    xh, _ = oracle.pdhg.pdhg_operator(sc.A, sc.c, sc.lx, sc.ux, sc.lc, sc.uc, np.zeros(3000),
                                      np.zeros(24), tau, sigma)
    bound = sigma * rel * (abs(sc.A) @ np.abs(2.0 * xh))
    ref = oracle.pdhg_solve(lp, opts, eta=eta, omega0=om)
    _, yi = _one_mixed_iteration(pkg, dev, lp, engine, eta, om, scaled)
    err = np.abs(yi - ref.y_iter) / sc.dr
    assert np.all(err <= bound + 1e-15 * np.max(np.abs(ref.y_iter / sc.dr)))
    # K1 (rows of A^T): 24 columns of 3,000 entries, warm-started y > 0
    A = rng.integers(1, 4, (3000, 24)).astype(float)
    b = A @ np.ones(24)
    lp = SimpleLP(A, rng.uniform(0.5, 1.5, 24), b, b, np.zeros(24), np.full(24, INF))
    sc = oracle.pdhg.Scaled(lp, opts)
    y0 = rng.uniform(0.5, 1.5, 3000)
    ref = oracle.pdhg_solve(lp, opts, eta=eta, omega0=om, y_init=y0)
    bound = tau * rel * (abs(sc.A).T @ np.abs(y0 / sc.dr))
    xi, _ = _one_mixed_iteration(pkg, dev, lp, engine, eta, om, scaled, y_init=y0)
    err = np.abs(xi - ref.x_iter) / sc.dc
    assert np.all(err <= bound + 1e-15 * np.max(np.abs(ref.x_iter / sc.dc)))
    assert np.max(np.abs(xi)) > 0 and np.max(np.abs(yi)) > 0


@pytest.mark.parametrize("engine", ENGINES)
def test_deterministic_reruns(pkg, dev, engine):
    lp = lpgen.general_structure(600, 1500, 4, nnz_target=9000)
    prob = pkg.Problem(lp, dev)
    prob.solve(max_iter=500, eps_rel=0.0, engine=engine)
    a = prob.iterate()
    prob.solve(max_iter=500, eps_rel=0.0, engine=engine)
    b = prob.iterate()
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("engine", ENGINES)
def test_degenerate_shapes(pkg, dev, engine):
    # no rows: each column goes to the bound its cost points to
    lp = SimpleLP(np.zeros((0, 3)), [1.0, -2.0, 0.0], [], [], [-1.0, 0.0, -3.0],
                  [4.0, 5.0, 3.0])
    prob = pkg.Problem(lp, dev)
    r = prob.solve(eps_rel=1e-9, engine=engine)
    assert r.termination == pkg.LP_OPTIMAL
    x, _, _ = prob.solution()
    assert np.allclose(x, [-1.0, 5.0, 0.0], atol=1e-8)
    # an empty row and an empty column kept (no presolve)
    lp = SimpleLP([[1.0, 0.0, 1.0], [0.0, 0.0, 0.0]], [1.0, 0.0, 2.0], [1.0, -1.0],
                  [1.0, 1.0], [0.0, 0.0, 0.0], [INF, 2.0, INF])
    prob = pkg.Problem(lp, dev)
    r = prob.solve(eps_rel=1e-9, engine=engine)
    assert r.termination == pkg.LP_OPTIMAL
    assert abs(r.primal_obj - 1.0) <= 1e-7


@pytest.mark.parametrize("engine", ENGINES)
def test_warm_start_from_solution_converges_at_first_check(pkg, dev, engine):
    lp = lpgen.c1_small()
    prob = pkg.Problem(lp, dev)
    r = prob.solve(x_init=lp.x_star, y_init=lp.y_star, engine=engine)
    assert r.termination == pkg.LP_OPTIMAL and r.iterations == 1


def test_resolve_after_other_options_matches_fresh_solve(pkg, dev):
    # a CUDA graph captured during an earlier solve must see the current
    # scaling: a re-solve behaves exactly like a solve on a fresh problem
    lp = lpgen.c1_small()
    fresh = pkg.Problem(lp, dev)
    r0 = fresh.solve(engine=1)
    x0, y0, _ = fresh.solution()
    prob = pkg.Problem(lp, dev)
    prob.solve(max_iter=50, eps_rel=0.0, step_size=0.05, primal_weight=1.3, engine=1)
    prob.solve(max_iter=700, ruiz_iters=3, pock_chambolle=0, engine=1)
    r = prob.solve(engine=1)
    assert r.termination == pkg.LP_OPTIMAL
    assert r.iterations == r0.iterations and r.restarts == r0.restarts
    x, y, _ = prob.solution()
    np.testing.assert_array_equal(x, x0)
    np.testing.assert_array_equal(y, y0)


def test_engines_agree_on_iterates(pkg, dev):
    # the cluster engine runs the grid engine's algorithm: after the same
    # number of iterations both hold the same point up to rounding order
    lp = lpgen.general_structure(900, 2200, 21, nnz_target=15000, one_sided=0.2)
    out = []
    for engine in ENGINES:
        prob = pkg.Problem(lp, dev)
        r = prob.solve(max_iter=200, eps_rel=0.0, engine=engine)
        out.append((r, prob.iterate(), prob.solution()))
        prob.close()
    (ra, ia, sa), (rb, ib, sb) = out
    assert ra.iterations == rb.iterations == 200
    assert ra.restarts == rb.restarts
    assert relerr(ia[0], ib[0]) <= 1e-9 and relerr(ia[1], ib[1]) <= 1e-9
    assert relerr(sa[0], sb[0]) <= 1e-9 and relerr(sa[1], sb[1]) <= 1e-9


@pytest.mark.parametrize("engine", ENGINES)
def test_rows_summing_to_zero_get_a_real_step(pkg, dev, engine):
    # A = [1, -1] (A 1 = 0): the step size comes from ||A~|| = sqrt(2) a, as in
    # the oracle, and the LP min x1 + x2, x1 - x2 = 0.5, 0 <= x <= 10 solves
    lp = SimpleLP([[1.0, -1.0]], [1.0, 1.0], [0.5], [0.5], [0.0, 0.0], [10.0, 10.0])
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=1, eps_rel=0.0))
    prob = pkg.Problem(lp, dev)
    r = prob.solve(max_iter=1, eps_rel=0.0, engine=engine)
    assert abs(r.eta - ref.eta) <= 1e-12 * ref.eta
    prob = pkg.Problem(lp, dev)
    r = prob.solve(engine=engine)
    assert r.termination == pkg.LP_OPTIMAL
    assert abs(r.primal_obj - 0.5) <= 1e-5


@pytest.mark.parametrize("engine", ENGINES)
def test_original_lp_check_re_solves_an_amplified_postsolve(pkg, dev, engine):
    # a fixed column shrinks every right-hand side 30x in the original LP:
    # the reduced solve at 1e-6 misses 1e-6 on the original, the check
    # re-solves at 1e-7 (warm-started) and the postsolved point meets it
    lp = lpgen.amplified_postsolve(seed=43)
    prob = pkg.Problem(lp, dev)
    prob.presolve()
    r0 = prob.solve(engine=engine, refine_original=0)
    assert r0.termination == pkg.LP_OPTIMAL and r0.refinements == 0
    x, y, _ = prob.postsolve()
    assert oracle.rel_kkt(lp, x, y)["rel_kkt"] > 2e-6
    r = prob.solve(engine=engine)
    assert r.termination == pkg.LP_OPTIMAL
    assert r.refinements >= 1 and r.iterations > r0.iterations
    x, y, _ = prob.postsolve()
    k = oracle.rel_kkt(lp, x, y)
    assert r.rel_kkt_original <= 1e-6 and k["rel_kkt"] <= 1e-6 * (1 + 1e-6)
    assert abs(k["rel_kkt"] - r.rel_kkt_original) <= 1e-6 * r.rel_kkt_original
    assert rel_obj(k["p"], lp.p_star) <= 1e-6
    # the oracle's pipeline (same reading) also needs a re-solve here
    ref = oracle_pipeline.solve_original(lp)
    assert ref.refinements >= 1 and ref.kkt["rel_kkt"] <= 1e-6
    assert rel_obj(k["p"], ref.kkt["p"]) <= 1e-6
    prob.close()


SHAPES = [(8, 512), (8, 2048), (16, 512), (16, 2048), (32, 512), (32, 2048), (64, 512),
          (64, 2048)]


@pytest.fixture(scope="module")
def powerlaw_lp():
    # row lengths from 1 to thousands and 20 columns of 2,500 entries: rows
    # of A and of A^T longer than 32 * run_max are segmented under every shape
    return lpgen.c3_powerlaw(seed=7, m=3000, n=8000, row_nnz_target=60000, n_dense=20,
                             dense_len=2500, kmax=6000)


@pytest.mark.parametrize("shape", SHAPES)
def test_every_tile_shape_matches_oracle(pkg, dev, powerlaw_lp, shape):
    # 130 iterations straddle the checks at 64 and 128, whose restart test and
    # primal-weight update read the segmented rows' own partial slots
    lp = powerlaw_lp
    eta, om = 0.02, 0.7
    prob = pkg.Problem(lp, dev)
    for iters in (40, 130):
        ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=iters, eps_rel=0.0), eta=eta,
                                omega0=om)
        r = prob.solve(max_iter=iters, eps_rel=0.0, step_size=eta, primal_weight=om, engine=1,
                       tile_run_max=shape[0], tile_nnz=shape[1])
        assert r.restarts == ref.restarts
        xi, yi = prob.iterate()
        assert relerr(xi, ref.x_iter) <= 1e-10 and relerr(yi, ref.y_iter) <= 1e-10
        assert abs(r.rel_kkt - ref.kkt["rel_kkt"]) <= 1e-9 * (1 + ref.kkt["rel_kkt"])
        tt = prob.tile_tuning()
        assert tt["shapes"][tt["A"]] == shape and tt["shapes"][tt["T"]] == shape
    # the step size (power iteration through the segmented rows) and omega_0
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=1, eps_rel=0.0))
    r = prob.solve(max_iter=1, eps_rel=0.0, engine=1, tile_run_max=shape[0], tile_nnz=shape[1])
    assert abs(r.eta - ref.eta) <= 1e-12 * ref.eta
    assert abs(r.omega - ref.omega0) <= 1e-12 * ref.omega0
    prob.close()


def test_shape_change_between_solves_matches_oracle(pkg, dev, powerlaw_lp):
    # run_max 8 segments every row over 256 entries, run_max 32 only those
    # over 1024: the second solve on the same upload must not sum the slots
    # the first plan's extra segmented rows left (step size, restart tests)
    lp = powerlaw_lp
    prob = pkg.Problem(lp, dev)
    prob.solve(max_iter=130, eps_rel=0.0, engine=1, tile_run_max=8, tile_nnz=512)
    ref = oracle.pdhg_solve(lp, oracle.Opts(max_iter=130, eps_rel=0.0))
    r = prob.solve(max_iter=130, eps_rel=0.0, engine=1, tile_run_max=32, tile_nnz=2048)
    assert abs(r.eta - ref.eta) <= 1e-12 * ref.eta
    assert r.restarts == ref.restarts
    xi, yi = prob.iterate()
    assert relerr(xi, ref.x_iter) <= 1e-10 and relerr(yi, ref.y_iter) <= 1e-10
    prob.close()


def test_autotuner_keeps_the_fastest_shape_and_caches_it(pkg, dev, powerlaw_lp):
    pkg.tile_cache_clear()
    prob = pkg.Problem(powerlaw_lp, dev)
    r1 = prob.solve(max_iter=300, eps_rel=0.0, engine=1)
    t1 = prob.tile_tuning()
    assert t1["measured"]
    assert len(t1["shapes"]) == len(SHAPES) and set(t1["shapes"]) == set(SHAPES)
    assert all(v > 0 for v in t1["ms_A"] + t1["ms_T"])
    assert t1["ms_A"][t1["A"]] == min(t1["ms_A"])
    assert t1["ms_T"][t1["T"]] == min(t1["ms_T"])
    x1, y1 = prob.iterate()
    # the same size class again: the cached choice, no measurement, and the
    # same iterates bit for bit (the measurement does not touch the solve)
    r2 = prob.solve(max_iter=300, eps_rel=0.0, engine=1)
    t2 = prob.tile_tuning()
    assert not t2["measured"] and (t2["A"], t2["T"]) == (t1["A"], t1["T"])
    x2, y2 = prob.iterate()
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(y1, y2)
    assert r1.restarts == r2.restarts
    # and the same as a solve given those shapes (A and A^T each its own)
    if t1["A"] == t1["T"]:
        sh = t1["shapes"][t1["A"]]
        prob.solve(max_iter=300, eps_rel=0.0, engine=1, tile_run_max=sh[0], tile_nnz=sh[1])
        x3, y3 = prob.iterate()
        np.testing.assert_array_equal(x1, x3)
        np.testing.assert_array_equal(y1, y3)
    prob.close()


def test_tile_shape_options_are_validated(pkg, dev):
    prob = pkg.Problem(lpgen.c1_small(), dev)
    with pytest.raises(pkg.LPError):
        prob.solve(max_iter=5, engine=1, tile_run_max=12, tile_nnz=512)
    with pytest.raises(pkg.LPError):
        prob.solve(max_iter=5, engine=1, tile_run_max=8, tile_nnz=1000)
    prob.close()
