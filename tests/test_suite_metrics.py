"""The presolve on/off suite's metrics (Sec. 4.3) on hand-checked values (CPU),
and one tiny suite instance end to end on the GPU."""
import math

import numpy as np
import pytest

import suite


def test_sgm_closed_forms():
    # equal times: the SGM is that time for any shift
    assert abs(suite.sgm([3.0] * 5, 1.0) - 3.0) <= 1e-12
    assert abs(suite.sgm([3.0] * 5, 10.0) - 3.0) <= 1e-12
    # (1 + 1)(3 + 1) = 8 -> sqrt(8) - 1
    assert abs(suite.sgm([1.0, 3.0], 1.0) - (math.sqrt(8.0) - 1.0)) <= 1e-12
    # zeros stay zero; a larger shift pulls the mean toward the arithmetic one
    assert suite.sgm([0.0, 0.0], 1.0) == 0.0
    t = [0.01, 0.1, 10.0, 100.0]
    g1, g10 = suite.sgm(t, 1.0), suite.sgm(t, 10.0)
    gm = math.exp(np.mean(np.log(t)))
    assert gm < g1 < g10 < np.mean(t)


def test_win_rate_and_classes():
    assert suite.win_rate([1.0, 2.0, 3.0, 4.0], [2.0, 2.0, 1.0, 5.0]) == 50.0
    assert suite.size_class(99_999) == "tiny"
    assert suite.size_class(100_000) == "small"
    assert suite.size_class(999_999) == "small"
    assert suite.size_class(1_000_000) == "medium"
    assert suite.size_class(10_000_000) == "large"


def test_instance_sizes_stay_in_their_class():
    for cls, nnz, seed in suite.instance_sizes(["small", "medium", "large"], 6):
        lo, hi = suite.CLASSES[cls]
        assert lo * 1.05 <= nnz <= hi / 1.2
    seeds = [s for _, _, s in suite.instance_sizes(["small", "medium"], 3)]
    assert len(set(seeds)) == len(seeds)


def test_summary_counts_failures_at_the_limit():
    recs = [
        {"t_off": 2.0, "ok_off": True, "t_on": 1.0, "ok_on": True, "t_presolve": 0.1,
         "t_reduced_solve": 0.9, "nnz": 100, "nnz_reduced": 80},
        {"t_off": 5.0, "ok_off": False, "t_on": 3.0, "ok_on": True, "t_presolve": 0.5,
         "t_reduced_solve": 2.5, "nnz": 100, "nnz_reduced": 60},
    ]
    s = suite.summarize(recs, time_limit=100.0)
    assert s["count_off"] == 1 and s["count_on"] == 2
    assert abs(s["sgm1_off"] - suite.sgm([2.0, 100.0], 1.0)) <= 1e-12
    assert abs(s["sgm1_on"] - suite.sgm([1.0, 3.0], 1.0)) <= 1e-12
    assert s["win_rate_pct"] == 100.0
    assert abs(s["nnz_ratio"] - 0.7) <= 1e-12
    assert abs(s["presolve_pct_of_reduced_solve"] - 0.5 * (100 * 0.1 / 0.9 + 100 * 0.5 / 2.5)) <= 1e-9


@pytest.mark.gpu
def test_suite_instance_both_arms_solve():
    import paper_2604_23951_gb300 as pkg

    pkg.load()
    dev = pkg.TorchDevice(0)
    lp = suite.make_instance(30_000, 123)
    rec = suite.run_instance(pkg, dev, lp, 1e-6, 60.0, pkg.LP_FP64)
    assert rec["ok_off"] and rec["ok_on"], rec
    assert rec["kkt_off"] <= 1e-6 and rec["kkt_on"] <= 1e-6
    assert rec["nnz_reduced"] < rec["nnz"]
