"""Presolve on/off suite reported with the paper's end-to-end metrics (Sec. 4).

Generated planted LPs in the paper's three size classes (small: 1e5-1e6
nonzeros, medium: 1e6-1e7, large: more than 1e7) are each solved on the GPU
twice through the library's public API:

* presolve off: create + solve of the original LP;
* presolve on:  create + host presolve + solve of the reduced LP (+ postsolve,
  timed separately; the paper's total is presolve + reduced solve).

Reported per class and over all instances (Sec. 4.3's metrics):

* count: instances solved to the tolerance within the time limit;
* SGM1 / SGM10: shifted geometric mean (prod (t_i + D))^(1/K) - D of the total
  time with shift D = 1 s and 10 s; an unsolved instance counts at the limit;
* win rate: percentage of instances whose total time with presolve is lower;
* presolve time as a percentage of the reduced solve time (Table 4), the
  reduced / original nnz ratio and the presolve time's arithmetic and
  geometric means (Table 2).

Each solution is checked on the original LP (host FP64 relative KKT error,
after postsolve for the presolve arm).  The instances are seeded synthetic
stand-ins for the paper's Mittelmann and MIPLIB sets: `lpgen.medium_structure`
(C2's row/column mix plus parallel rows and slack column singletons), with
nnz drawn log-uniformly inside each class and m = nnz / 25, n = 2.5 m.

    python suite.py --per-class 4 --classes small,medium,large --out suite.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CLASSES = {"small": (1e5, 1e6), "medium": (1e6, 1e7), "large": (1e7, 2e7)}
SUITE_SEED = 2604_23951 + 40


def sgm(times, shift: float) -> float:
    """Shifted geometric mean (prod (t_i + shift))^(1/K) - shift."""
    t = np.asarray(times, dtype=np.float64)
    if t.size == 0:
        return float("nan")
    return float(np.exp(np.mean(np.log(t + shift))) - shift)


def win_rate(t_on, t_off) -> float:
    """Percentage of instances whose total time with presolve is lower."""
    a, b = np.asarray(t_on, np.float64), np.asarray(t_off, np.float64)
    if a.size == 0:
        return float("nan")
    return float(100.0 * np.mean(a < b))


def size_class(nnz: int) -> str:
    if nnz < 1e5:
        return "tiny"
    if nnz < 1e6:
        return "small"
    if nnz < 1e7:
        return "medium"
    return "large"


def instance_sizes(classes, per_class: int, seed: int = SUITE_SEED):
    """(class, nnz target, seed) per instance; nnz log-uniform in the class."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, name in enumerate(classes):
        lo, hi = CLASSES[name]
        for j in range(per_class):
            # the planted copies add ~10% nonzeros: aim inside the class
            nnz = float(np.exp(rng.uniform(math.log(lo * 1.05), math.log(hi / 1.2))))
            out.append((name, int(nnz), seed + 1000 * ci + j))
    return out


def make_instance(nnz_target: int, seed: int):
    import lpgen

    m = max(int(nnz_target / 25), 8)
    n = int(2.5 * m)
    return lpgen.medium_structure(m, n, seed, nnz_target=nnz_target)


def _kkt_original(pkg, lp, x, y) -> float:
    host = pkg.Problem(lp, None)
    try:
        return float(host.rel_kkt(x, y)["rel_kkt"])
    finally:
        host.close()


def run_instance(pkg, dev, lp, eps: float, time_limit: float, precision: int,
                 rules: int | None = None) -> dict:
    """Both arms on one LP; times are wall seconds around the API calls."""
    import torch

    rec = {"m": int(lp.m), "n": int(lp.n), "nnz": int(lp.nnz)}
    # presolve off
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = pkg.Problem(lp, dev)
    r = p.solve(eps_rel=eps, time_limit_s=time_limit, precision=precision)
    torch.cuda.synchronize()
    t_off = time.perf_counter() - t0
    x, y, _ = p.solution()
    p.close()
    rec.update(t_off=t_off, ok_off=bool(r.termination == pkg.LP_OPTIMAL),
               iters_off=int(r.iterations), kkt_off=_kkt_original(pkg, lp, x, y))
    # presolve on
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = pkg.Problem(lp, dev)
    t1 = time.perf_counter()
    info = p.presolve(enable=pkg.LP_RULE_ALL if rules is None else rules)
    t_pre = time.perf_counter() - t1
    m2, n2, nnz2 = p.dims()
    decided = info.status in (1, 2)  # presolve proved infeasible / unbounded
    if decided:
        ok_on, iters_on = False, 0
    elif m2 > 0 or n2 > 0:
        r = p.solve(eps_rel=eps, time_limit_s=time_limit, precision=precision)
        ok_on = bool(r.termination == pkg.LP_OPTIMAL)
        iters_on = int(r.iterations)
    else:
        ok_on, iters_on = info.status == 3, 0  # LP_PRESOLVE_SOLVED
    torch.cuda.synchronize()
    t_on = time.perf_counter() - t0
    t2 = time.perf_counter()
    kkt_on = float("inf")
    if not decided:
        x, y, _ = p.postsolve()
        kkt_on = _kkt_original(pkg, lp, x, y)
    t_post = time.perf_counter() - t2
    p.close()
    rec.update(t_on=t_on, t_presolve=t_pre, t_reduced_solve=t_on - t_pre, t_postsolve=t_post,
               ok_on=ok_on, iters_on=iters_on, nnz_reduced=int(nnz2), presolve_status=info.status,
               kkt_on=kkt_on)
    rec["ok_off"] = rec["ok_off"] and rec["kkt_off"] <= eps
    rec["ok_on"] = rec["ok_on"] and rec["kkt_on"] <= eps
    return rec


def summarize(recs, time_limit: float) -> dict:
    """The paper's metrics over a list of run_instance records."""
    if not recs:
        return {}
    t_off = [r["t_off"] if r["ok_off"] else time_limit for r in recs]
    t_on = [r["t_on"] if r["ok_on"] else time_limit for r in recs]
    pre = [r["t_presolve"] for r in recs]
    return {
        "instances": len(recs),
        "count_off": sum(r["ok_off"] for r in recs),
        "count_on": sum(r["ok_on"] for r in recs),
        "sgm1_off": sgm(t_off, 1.0), "sgm1_on": sgm(t_on, 1.0),
        "sgm10_off": sgm(t_off, 10.0), "sgm10_on": sgm(t_on, 10.0),
        "win_rate_pct": win_rate(t_on, t_off),
        "presolve_pct_of_reduced_solve": float(np.mean(
            [100.0 * r["t_presolve"] / max(r["t_reduced_solve"], 1e-12) for r in recs])),
        "nnz_ratio": float(np.mean([r["nnz_reduced"] / r["nnz"] for r in recs])),
        "presolve_am_s": float(np.mean(pre)),
        "presolve_gm_s": float(np.exp(np.mean(np.log(np.maximum(pre, 1e-12))))),
    }


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--classes", default="small,medium,large")
    ap.add_argument("--per-class", type=int, default=4)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--time-limit", type=float, default=120.0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--seed", type=int, default=SUITE_SEED)
    ap.add_argument("--propagation", action="store_true",
                    help="presolve also runs primal propagation (opt-in explorer)")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)

    import torch

    import paper_2604_23951_gb300 as pkg

    if not torch.cuda.is_available():
        print("suite.py needs a CUDA device", file=sys.stderr)
        return 2
    pkg.load()
    dev = pkg.TorchDevice(0)
    prec = pkg.LP_FP64 if args.precision == "fp64" else pkg.LP_MIXED
    classes = [c for c in args.classes.split(",") if c]
    # warm-up: context, allocator and kernels loaded before the first timing
    warm = make_instance(20_000, args.seed - 1)
    run_instance(pkg, dev, warm, args.eps, args.time_limit, prec)
    recs = []
    for cls, nnz, seed in instance_sizes(classes, args.per_class, args.seed):
        t0 = time.perf_counter()
        lp = make_instance(nnz, seed)
        t_gen = time.perf_counter() - t0
        rules = pkg.LP_RULE_ALL | (pkg.LP_RULE_PRIMAL_PROPAGATION if args.propagation else 0)
        rec = run_instance(pkg, dev, lp, args.eps, args.time_limit, prec, rules)
        rec.update(target_class=cls, size_class=size_class(rec["nnz"]), seed=seed,
                   t_generate=t_gen)
        recs.append(rec)
        print(json.dumps({k: (round(v, 4) if isinstance(v, float) and k.startswith("t_") else v)
                          for k, v in rec.items()}), flush=True)
        del lp
    out = {"eps_rel": args.eps, "time_limit_s": args.time_limit, "precision": args.precision,
           "propagation": bool(args.propagation),
           "gpu": torch.cuda.get_device_name(0), "records": recs,
           "summary": {c: summarize([r for r in recs if r["size_class"] == c], args.time_limit)
                       for c in ("small", "medium", "large")}}
    out["summary"]["all"] = summarize(recs, args.time_limit)
    print(json.dumps(out["summary"]), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
