#!/usr/bin/env python
"""Benchmark: time to relative KKT error 1e-6 on a planted LP, on GB300.

Default workload: the large planted LP with m = 2M rows, n = 5M columns and
~50M nonzeros (power-law row lengths up to 10k plus 5,000 columns of 2,000
entries; seeded, synthetic).  One step = one full device solve in FP64
(GPU scaling, power-iteration step size, restarted reflected Halpern PDHG to
rel-KKT <= 1e-6) with the LP resident in HBM; the same LP is then solved once
in the mixed precision and reported beside it with its per-instance
difference.  `e2e` times the whole C-ABI path from host buffers (lp_create,
lp_presolve for c2, lp_solve with its H2D upload, lp_postsolve with the D2H of
the solution).

Prints ONE JSON line (rank 0).  Under torchrun the single-LP workloads
(c1, c2, c3) run one replica per rank (no collective on the data path;
replicas only) and report the slowest rank's time; the batch (c4) and
serving (c5) workloads scale weakly: every rank solves its own seeded batch
or stream (rank 0 the configured one) and the value counts all ranks' LPs
over the slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3|c2|c1|c4|c5] [--precision fp64|mixed]
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel-KKT 1e-6 (s); SpMV HBM GB/s vs peak; batched LPs/s with p50/p99"

# Iterations to rel-KKT 1e-6 on each seeded workload (FP64) that the
# reference arm extrapolates its timed oracle sample with: the oracle's own
# count where it was run to completion (c1: 1217; c2, see ORACLE_C2_FULL),
# else the device solve's count (c3: a full oracle run would take about 15
# hours; the two follow the same iteration).
ITERS_TO_TOL = {"c2": 11841, "c1": 1217, "c3": 51905}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c3", choices=["c3", "c2", "c1", "c4", "c5"])
    p.add_argument("--requests", type=int, default=96, help="c5: stream length")
    p.add_argument("--lps", type=int, default=512,
                   help="c4: LPs in the batch (512 is the configuration; fewer for profiling)")
    p.add_argument("--rate", type=float, default=200.0, help="c5: arrivals per second")
    p.add_argument("--sweep", default="2,4,8",
                   help="c5: arrival rates (req/s) at which the first --sweep-count requests "
                        "are served again ('' for none)")
    p.add_argument("--sweep-count", type=int, default=24)
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--solo-nnz", type=int, default=0,
                   help="c4/c5: nonzeros from which a request runs the single-LP path (0: default)")
    p.add_argument("--solo-max", type=int, default=-1, help="c4/c5: concurrent solo requests")
    p.add_argument("--propagation", action="store_true",
                   help="c2/c5: presolve also runs primal propagation (opt-in explorer)")
    p.add_argument("--infeas-every", type=int, default=-1,
                   help="infeasibility test every N-th check (0: off; -1: library default)")
    p.add_argument("--launch-ms", type=float, default=0.0,
                   help="c4/c5: device time budget of one bucket launch (0: default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-mixed", action="store_true",
                   help="c2/c3: skip the solve in the other precision")
    p.add_argument("--scale", type=float, default=1.0,
                   help="c2/c3: generate the workload at this fraction of its size "
                        "(profiling captures of a smaller case; not a bench line)")
    p.add_argument("--profile-iters", type=int, default=0,
                   help="ncu capture command: one solve capped at this many iterations, "
                        "no timing and no JSON line")
    return p.parse_args()


def make_workload(name, scale=1.0):
    import lpgen

    if name == "c1":
        return lpgen.c1_small(), "planted LP 200 x 400, ~2,000 nnz, equality rows, x >= 0"
    if name == "c3":
        if scale != 1.0:
            s = float(scale)
            lp = lpgen.c3_powerlaw(m=int(2_000_000 * s), n=int(5_000_000 * s),
                                   row_nnz_target=int(40_000_000 * s),
                                   n_dense=max(1, int(5_000 * s)))
            return lp, f"planted LP C3 structure at scale {s:g} ({lp.m} x {lp.n}, {lp.nnz} nnz)"
        return lpgen.c3_powerlaw(), ("planted LP 2M x 5M, ~50M nnz, power-law rows + 5,000 "
                                     "dense columns, box bounds")
    if scale != 1.0:
        lp = lpgen.c2_presolvable(scale=float(scale))
        return lp, f"presolvable planted LP C2 structure at scale {scale:g}"
    return lpgen.c2_presolvable(), ("presolvable planted LP 200k x 500k, ~5M nnz "
                                    "(lognormal rows, 60% eq / 40% ranged, singleton, "
                                    "doubleton, fixed, mixed bounds)")


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [q.strip() for q in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# helpers


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values (the job's time), or x alone."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_share(rank: int, per_rank: int) -> int:
    """First item of rank's share of a batch workload scaled weakly: rank r
    solves items r * per_rank .. (r + 1) * per_rank - 1 of the seeded
    sequence, so rank 0 always solves the configuration's own batch."""
    return rank * per_rank


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def presolve_rules(pkg, args):
    """presolve rule mask: the default set, plus primal propagation if asked"""
    return pkg.LP_RULE_ALL | (pkg.LP_RULE_PRIMAL_PROPAGATION if args.propagation else 0)


def solver_kw(args):
    """lp_solve_opts fields set on the command line"""
    return {"infeas_every": args.infeas_every} if args.infeas_every >= 0 else {}


def iter_bytes(m, n, nnz, fp32):
    """Algorithmic bytes of one PDHG iteration (K1 + K2): both matrices'
    values and indices once, row offsets, each gathered vector once, and the
    epilogues' vectors (K1 reads x, x0, c, l, u and writes x and xbar; K2
    reads y, y0, l, u and writes y).  The mixed SpMV streams FP32 values and
    gathers x-bar and y as 8-byte float pairs, which K2 also writes for y."""
    sv = 4 if fp32 else 8
    k1 = nnz * (sv + 4) + 4 * (n + 1) + 8 * m + 8 * 6 * n + 8 * n
    k2 = nnz * (sv + 4) + 4 * (m + 1) + 8 * n + 8 * 5 * m + (8 * m if fp32 else 0)
    return k1 + k2


def tile_summary(srv):
    """The batched tile-shape autotuner's table: per (m bucket, row-length
    bucket) the chosen shape as (entries per lane, nonzeros per tile), or
    null while the class is still trying, and its sample count."""
    out = []
    for c in srv.tile_tuning():
        ch = c["chosen"]
        shape = None if ch < 0 else [(8, 16, 32)[ch // 2], 2048 if ch & 1 else 512]
        out.append({"class": [c["m_bucket"], c["len_bucket"]], "shape": shape,
                    "samples": sum(c["samples"])})
    return out


def fifo_latencies(arrivals, services):
    """arrival-to-completion times when requests are served one at a time in
    arrival order with the given service times"""
    out, free_at = [], 0.0
    for a, sv in zip(arrivals, services):
        free_at = max(free_at, a) + sv
        out.append(free_at - a)
    return out


def term_hist(codes):
    """{termination code: count} (0 optimal, 1 iteration limit, 2 time limit,
    3 numerical, 4 infeasible, 5 unbounded, 6 cancelled)"""
    h = {}
    for c in codes:
        h[str(int(c))] = h.get(str(int(c)), 0) + 1
    return h


def kernel_source_hash():
    """Hash of the source K1 / K2 are built from: the engine, epilogue, state
    and layout files, and in solver.cu the block-size constants and the text
    from the k_primal template through k_dual (other kernels there do not
    change the profiled launches)."""
    csrc = os.path.join(ROOT, "paper_2604_23951_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("device_common.cuh", "spmv_warp.cuh", "pdhg_epi.cuh", "pdhg_state.cuh",
              "layout.cpp", "layout.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "solver.cu"), "r") as fh:
        src = fh.read()
    a = src.index("constexpr int kBlock")
    h.update(src[a:src.index("\n\n", a)].encode())
    a = src.index("__global__ void __launch_bounds__(kBlock, IterBlocks<T>::value) k_primal(")
    b = src.index("__global__ void __launch_bounds__(kBlock, kMinBlocks) k_kkt_rows(")
    h.update(src[a:b].encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, precision: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[f"{kernel}/{workload}/{precision}"]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


def host_cpu():
    """(model name, logical cores) of this host"""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.startswith(("Model name", "Vendor ID")) and ":" in ln:
                    v = ln.split(":", 1)[1].strip()
                    model = v if model is None else f"{model} {v}"
        except Exception:
            pass
    if model is None:
        import platform

        model = platform.processor() or platform.machine()
    return model, os.cpu_count()


def oracle_sample(lp, n_iter_gpu, workload, iters=3):
    """The oracle as it stands on this host (one thread), on a bounded sample:
    presolve (C2), one Ruiz pass and one power-iteration step (each scaled to
    the 10 + 1 passes and 100 steps of the set-up), and `iters` PDHG
    iterations with the step size and weight given (the set-up's cost is
    counted above); extrapolated to n_iter_gpu iterations.  Returns (seconds,
    sample description, CPU seconds spent)."""
    import numpy as np

    import oracle
    from oracle import pdhg as P
    from oracle import presolve as PS

    spent = time.perf_counter()
    t0 = time.perf_counter()
    pres = PS.presolve(lp) if workload == "c2" else None
    t_pre = time.perf_counter() - t0
    red = pres.reduced if pres is not None else lp
    A = P.csr_of(red)
    t0 = time.perf_counter()
    P.ruiz_pc_scaling(A, 1, False)
    t_ruiz = time.perf_counter() - t0
    t0 = time.perf_counter()
    v = np.full(red.n, 1.0)
    A.T @ (A @ v)
    t_pow = time.perf_counter() - t0
    base = dict(eps_rel=0.0, ruiz_iters=0, pock_chambolle=False, infeas_every=0)
    t0 = time.perf_counter()
    oracle.pdhg_solve(red, oracle.Opts(max_iter=1, **base), eta=0.01, omega0=1.0)
    t_1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pdhg_solve(red, oracle.Opts(max_iter=1 + iters, **base), eta=0.01, omega0=1.0)
    per_iter = max(time.perf_counter() - t0 - t_1, 0.0) / iters
    setup = 11 * t_ruiz + 100 * t_pow + t_1
    est = t_pre + setup + per_iter * max(n_iter_gpu - 1, 0)
    model, nproc = host_cpu()
    sample = (f"EXTRAPOLATION: oracle (NumPy/SciPy, 1 thread) on {model} ({nproc} logical "
              f"cores): presolve {t_pre:.2f} s measured; set-up = 11 x one Ruiz/Pock-Chambolle "
              f"pass ({t_ruiz:.2f} s) + 100 x one power step ({t_pow:.2f} s) + first iteration "
              f"({t_1:.2f} s); {iters} timed PDHG iterations ({per_iter:.3f} s each) x "
              f"{n_iter_gpu} iterations (the device solve's count)")
    return est, sample, time.perf_counter() - spent


# The oracle run to completion once on the presolved 200k x 500k workload,
# one thread of an 8-core Xeon @ 2.7 GHz: presolve 19.3 s, PDHG 554.9 s,
# 11,841 iterations (46.9 ms each), 12 restarts, rel-KKT 7.35e-7 on the
# reduced and 7.05e-7 on the original LP (no re-solve needed); the device's
# FP64 solve of the same LP takes 12,161 iterations.
ORACLE_C2_FULL = {"presolve_s": 19.30, "solve_s": 554.91, "iterations": 11841,
                  "restarts": 12, "rel_kkt_original": 7.05e-7,
                  "host": "Intel Xeon @ 2.70GHz, 8 logical cores, 1 thread"}


# ---------------------------------------------------------------------------
# arms


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the
    workload, extrapolated as in oracle_sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    lp, desc = make_workload(args.workload, args.scale)
    n_iter = ITERS_TO_TOL[args.workload]
    vals, sample, spent = [], None, 0.0
    for step in range(args.warmup + args.steps):
        est, sample, sp = oracle_sample(lp, n_iter, args.workload)
        spent += sp
        if step >= args.warmup:
            vals.append(est)
    value = statistics.mean(vals)
    model, nproc = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": sample, "host_cpu": model, "host_logical_cores": nproc,
                         "cpu_seconds_spent": round(spent, 1)},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2604_23951_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    pkg.load()
    lp, desc = make_workload(args.workload, args.scale)
    dev = pkg.TorchDevice(local)
    prec = pkg.LP_MIXED if args.precision == "mixed" else pkg.LP_FP64
    prob = pkg.Problem(lp, dev)
    info = prob.presolve(enable=presolve_rules(pkg, args)) if args.workload == "c2" else None
    prob.upload()
    m, n, nnz = prob.dims()
    if args.profile_iters > 0:
        r = prob.solve(precision=prec, max_iter=args.profile_iters, eps_rel=0.0)
        print(f"profile case: {args.workload} {args.precision} m={m} n={n} nnz={nnz} "
              f"iterations={r.iterations} launches={r.kernel_launches}", flush=True)
        return 0
    for _ in range(args.warmup):
        r = prob.solve(precision=prec, **solver_kw(args))
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    stream = dev.stream
    # each timed solve starts with L2 flushed (a 256 MiB write, outside the
    # timed events); the step time is the solve between events on its stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    results = []
    elapsed = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        results.append(prob.solve(precision=prec, **solver_kw(args)))
        ev1.record(stream)
        ev1.synchronize()
        elapsed += ev0.elapsed_time(ev1) / 1e3
    barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(elapsed, dist, f"cuda:{local}")
    value = elapsed / args.steps
    r = results[-1]
    tiles = prob.tile_tuning()
    launches = int(sum(x.kernel_launches for x in results))
    # the other precision on the same LP: time to 1e-6 and, per instance,
    # its objective and rel-KKT against this solve's
    other = None
    if not args.no_mixed and args.workload in ("c2", "c3"):
        oprec = pkg.LP_FP64 if prec == pkg.LP_MIXED else pkg.LP_MIXED
        prob.solve(precision=oprec, max_iter=256, eps_rel=0.0)  # shape measurement
        with torch.cuda.stream(stream):
            flush.fill_(1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ro = prob.solve(precision=oprec, **solver_kw(args))
        ev1.record(stream)
        ev1.synchronize()
        t_o = ev0.elapsed_time(ev1) / 1e3
        fp64 = r if prec == pkg.LP_FP64 else ro
        mix = ro if prec == pkg.LP_FP64 else r
        other = {"precision": "mixed" if oprec == pkg.LP_MIXED else "fp64", "value": t_o,
                 "unit": "s", "iterations": int(ro.iterations),
                 "fp32_iterations": int(ro.fp32_iterations), "rel_kkt": ro.rel_kkt,
                 "termination": int(ro.termination),
                 "mixed_vs_fp64": {
                     "objective_rel_diff": abs(mix.primal_obj - fp64.primal_obj)
                     / (1 + abs(fp64.primal_obj)),
                     "rel_kkt_mixed": mix.rel_kkt, "rel_kkt_fp64": fp64.rel_kkt,
                     "time_ratio_mixed_over_fp64": (t_o / value if oprec == pkg.LP_MIXED
                                                    else value / t_o)},
                 "note": "one solve of the same LP (L2 flushed before it); per-instance "
                         "objective difference against the FP64 solve"}
    # per-kernel timing (CUDA events, cold L2) for the roofline: the grid
    # engine's K1 / K2 in the bench precision, set up by a short solve
    prob.solve(precision=prec, max_iter=128, eps_rel=0.0, engine=pkg.LP_ENGINE_GRID)
    prof = prob.profile_kernels(reps=10)
    peak, peak_kind = peaks()
    cand = {"primal": (prof["primal_ms"], prof["primal_bytes"]),
            "dual": (prof["dual_ms"], prof["dual_bytes"])}
    dom = max(cand, key=lambda k: cand[k][0])
    ms, byt = cand[dom]
    achieved = byt / (ms * 1e-3) / 1e9
    kname = {"primal": "k_primal", "dual": "k_dual"}[dom]
    traffic = ncu_traffic(kname, args.workload, args.precision)
    # end to end through the C ABI from host buffers
    barrier()
    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(1, min(args.steps, 3 if args.workload != "c3" else 1))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = pkg.Problem(lp, dev)
        if args.workload == "c2":
            p2.presolve(enable=presolve_rules(pkg, args))
        r2 = p2.solve(precision=prec, **solver_kw(args))
        x, y, z = p2.postsolve()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        m2, n2, nnz2 = p2.dims()
        h2d = 2 * nnz2 * 12 + 4 * (m2 + 1) + 4 * (n2 + 1) + 8 * (3 * n2 + 2 * m2)
        d2h = 8 * (3 * n2 + 2 * m2)
        p2.close()
    e2e = statistics.mean(e2e_times)
    obj_err = abs(r2.primal_obj - lp.p_star) / (1 + abs(lp.p_star))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, sample, spent = oracle_sample(lp, int(r.iterations), args.workload)
        model, nproc = host_cpu()
        cpu = {"value": est, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
               "host_cpu": model, "host_logical_cores": nproc,
               "cpu_seconds_spent": round(spent, 2)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == pkg.LP_FP64 else "f32 SpMV / f64 iterates",
            "data": "synthetic",
            "config": {
                "workload": desc, "m": int(lp.m), "n": int(lp.n), "nnz": int(lp.nnz),
                "reduced": {"m": m, "n": n, "nnz": nnz} if info is not None else None,
                "presolve_s": round(info.seconds, 4) if info is not None else None,
                "precision": args.precision, "parallelism": f"replicas{world}",
                "l2": "L2 flushed (256 MiB write) before each timed solve",
            },
            "iterations": int(r.iterations), "restarts": int(r.restarts),
            "termination": int(r.termination), "rel_kkt": r.rel_kkt,
            "rel_kkt_original_after_postsolve": r2.rel_kkt_original,
            "refinements": int(r2.refinements),
            "objective_rel_err_vs_planted": obj_err,
            "us_per_iteration": 1e6 * r.t_solve_s / max(1, r.iterations),
            "tile_shapes": {"A": tiles["shapes"][tiles["A"]], "AT": tiles["shapes"][tiles["T"]]},
            "other_precision": other,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                         "peak_kind": peak_kind, "kernel_ms": ms, "algorithmic_bytes": byt,
                         "other_kernels": {k: {"ms": v[0], "GB/s": v[1] / (v[0] * 1e-3) / 1e9}
                                           for k, v in cand.items()}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _gen_c5(req):
    import lpgen  # noqa: F401

    return req.make()


def run_batch(args):
    """c4: 512 planted LPs in one persistent batched launch (LPs/s, p50/p99);
    c5: a Poisson request stream served with continuous batching."""
    import numpy as np
    import torch

    import lpgen
    import oracle
    import paper_2604_23951_gb300 as pkg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.load()
    dev = pkg.TorchDevice(local)
    prec = pkg.LP_MIXED if args.precision == "mixed" else pkg.LP_FP64
    if args.workload == "c4":
        count = max(1, min(512, args.lps))
        lps = lpgen.c4_batch(count, first=weak_share(rank, count))
        # device budget: the packed slots with room to spare (~2.2 GB for 512)
        budget = int(max(256 << 20, 3 * sum(lp.nnz * 48 + (lp.m + lp.n) * 200 for lp in lps)))
        desc = (f"{len(lps)} planted LPs, m log-uniform [100, 20k], n = 2m, 4-30 nnz/row, "
                "equality, x >= 0, all submitted at once (16 submitting threads, server "
                "worker thread)")

        from concurrent.futures import ThreadPoolExecutor

        nsub = min(16, os.cpu_count() or 4)

        def one_step():
            probs = [pkg.Problem(lp, dev) for lp in lps]
            # a worker thread drives the device while the requests are still
            # being packed; several host threads submit (the packing of a
            # request runs on its submitting thread)
            srv = pkg.Server(budget, dev, worker=True, precision=prec, **solver_kw(args))
            srv.tune(args.solo_nnz, args.solo_max, args.launch_ms)
            t0 = time.perf_counter()
            with ThreadPoolExecutor(nsub) as ex:
                tickets = list(ex.map(srv.submit, probs))
            t_sub = time.perf_counter() - t0
            res = {}
            pending = list(tickets)
            while pending:
                left = []
                for t in pending:
                    got = srv.poll(t)
                    if got is None:
                        left.append(t)
                    else:
                        res[t] = got
                pending = left
                if pending:
                    time.sleep(0.0005)
            el = time.perf_counter() - t0
            lat = [res[t][0].t_total_s for t in tickets]
            errs = [abs(res[t][0].primal_obj - lp.p_star) / (1 + abs(lp.p_star))
                    for t, lp in zip(tickets, lps)]
            opt = sum(1 for t in tickets if res[t][0].termination == 0)
            st = srv.stats()
            st["terminations"] = term_hist(res[t][0].termination for t in tickets)
            st["submit_s"] = t_sub
            st["submit_threads"] = nsub
            st.update(srv.graph_stats())
            st["tile_classes"] = tile_summary(srv)
            srv.close()
            per = [(int(res[t][0].iterations), int(res[t][0].fp32_iterations),
                    res[t][0].primal_obj, res[t][0].rel_kkt) for t in tickets]
            return el, lat, errs, opt, st, per

        for _ in range(args.warmup):
            one_step()
        clocks = ClockSampler(local)
        clocks.start()
        steps = [one_step() for _ in range(args.steps)]
        clk = clocks.stop()
        # weak scaling: every rank solves its own batch; the job's time is the
        # slowest rank's, and the value counts every rank's LPs
        el = max_over_ranks(statistics.mean(s_[0] for s_ in steps), dist, f"cuda:{local}")
        lat = steps[-1][1]
        value = world * len(lps) / el
        per = steps[-1][5]
        # the batch as a roofline: the algorithmic bytes of every slot
        # iteration (each LP's FP32-SpMV iterations and FP64 ones) over the
        # batch's wall time, against the measured copy bandwidth
        peak, peak_kind = peaks()
        tot_bytes = sum(iter_bytes(lp.m, lp.n, lp.nnz, True) * f32
                        + iter_bytes(lp.m, lp.n, lp.nnz, False) * (its - f32)
                        for lp, (its, f32, _, _) in zip(lps, per))
        achieved = tot_bytes / statistics.mean(s_[0] for s_ in steps) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_batch",
                "peak_kind": peak_kind,
                "note": "algorithmic bytes of every slot-iteration of the batch (K1 + K2 bytes "
                        "at each iteration's SpMV precision) / the batch's wall time, which also "
                        "holds submission, set-up, checks and the host loop"}
        # comparator: the same LPs solved singly in plain FP64 (lp_solve, one
        # after another), on every 16th LP of the batch; per instance the
        # batch's (mixed) objective against that FP64 solve
        idx = list(range(0, len(lps), 16)) if len(lps) >= 16 else [0]
        t0 = time.perf_counter()
        diffs = []
        for j in idx:
            p = pkg.Problem(lps[j], dev)
            rs = p.solve(precision=pkg.LP_FP64)
            p.close()
            diffs.append({"item": j, "m": int(lps[j].m),
                          "objective_rel_diff": abs(per[j][2] - rs.primal_obj)
                          / (1 + abs(rs.primal_obj)),
                          "rel_kkt_batch": per[j][3], "rel_kkt_fp64": rs.rel_kkt})
        ts = time.perf_counter() - t0
        single = {"LPs_per_s": len(idx) / ts, "sample": f"{len(idx)} of the 512 LPs (every 16th), "
                  f"each lp_create + lp_solve (FP64) + lp_destroy, one after another ({ts:.1f} s)"}
        od = [d["objective_rel_diff"] for d in diffs]
        vs_fp64 = {"instances": len(diffs), "objective_rel_diff_max": max(od),
                   "objective_rel_diff_median": float(np.median(od)), "per_instance": diffs}
        cpu = None
        vs_oracle = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            pick = list(range(0, len(lps), max(1, len(lps) // 8)))[:8]
            t0 = time.perf_counter()
            vs_oracle = []
            for j in pick:
                ro = oracle.pdhg_solve(lps[j])
                vs_oracle.append({"item": j, "objective_rel_diff": abs(per[j][2] - ro.kkt["p"])
                                  / (1 + abs(ro.kkt["p"])), "rel_kkt_oracle": ro.kkt["rel_kkt"]})
            tc = time.perf_counter() - t0
            model, nproc = host_cpu()
            cpu = {"value": len(pick) / tc, "unit": "LPs/s", "cores": 1, "kind": "oracle",
                   "sample": f"oracle solves of {len(pick)} of the 512 LPs (every 64th) to "
                             f"rel-KKT 1e-6, sequential ({tc:.1f} s)",
                   "host_cpu": model, "host_logical_cores": nproc}
        line = {
            "metric": METRIC, "value": value, "unit": "LPs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == pkg.LP_FP64 else "f32 SpMV / f64 iterates",
            "data": "synthetic",
            "config": {"workload": desc, "lps": len(lps), "precision": args.precision,
                       "sum_nnz": int(sum(lp.nnz for lp in lps)), "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (~2 GB resident)"},
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "optimal": steps[-1][3], "max_objective_rel_err_vs_planted": max(steps[-1][2]),
            "vs_fp64_per_instance": vs_fp64, "vs_oracle_per_instance": vs_oracle,
            "roofline": roof,
            "single_fp64": single,
            "server_stats": steps[-1][4], "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "LPs/s",
                    "h2d_bytes_per_step": int(sum(lp.nnz * 24 + (lp.m + lp.n) * 24 for lp in lps)),
                    "d2h_bytes_per_step": int(sum((2 * lp.n + lp.m) * 8 for lp in lps))},
            "e2e_note": "value already includes the H2D of every request (submit) and the D2H "
                        "of every answer (poll)",
            "clocks": clk, "gpu_launches": steps[-1][4]["launches"],
        }
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    # ---- c5: serving stream --------------------------------------------------
    import multiprocessing as mp

    # weak scaling: every rank serves its own stream (rank 0: the configured one)
    reqs = lpgen.c5_stream(count=args.requests, rate=args.rate,
                           seed=lpgen.BASE_SEED + 5 + 1_000_003 * rank)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        lps = pool.map(_gen_c5, reqs)
    desc = (f"Poisson stream: {len(reqs)} planted LPs at {args.rate:g} req/s, nnz log-uniform "
            f"[1e3, 1e7], presolvable structure, 150 GB HBM budget")

    def serve(arrivals, lps_):
        """Serve lps_ arriving at the given times (s from the start); returns
        (elapsed, {j: (latency, result)}, server stats)."""
        srv = pkg.Server(int(150e9), dev, worker=True, precision=prec, **solver_kw(args))
        srv.tune(args.solo_nnz, args.solo_max, args.launch_ms)
        probs = [None] * len(lps_)
        tickets = [None] * len(lps_)
        arr = [None] * len(lps_)
        t0 = time.perf_counter()
        done = {}
        import threading as th

        def submitter():
            for j, (a, lp) in enumerate(zip(arrivals, lps_)):
                while time.perf_counter() - t0 < a:
                    time.sleep(0.0005)
                arr[j] = time.perf_counter()
                p = pkg.Problem(lp, dev)
                p.presolve(enable=presolve_rules(pkg, args))
                probs[j] = p
                tickets[j] = srv.submit(p)

        sub = th.Thread(target=submitter)
        sub.start()
        while len(done) < len(lps_):
            for j in range(len(lps_)):
                if j in done or tickets[j] is None:
                    continue
                got = srv.poll(tickets[j])
                if got is not None:
                    probs[j].postsolve()
                    done[j] = (time.perf_counter() - arr[j], got[0])
            time.sleep(0.001)
        sub.join()
        el = time.perf_counter() - t0
        st = srv.stats()
        st.update(srv.graph_stats())
        st["tile_classes"] = tile_summary(srv)
        srv.close()
        return el, done, st

    arrivals = [rq.arrival_s for rq in reqs]
    for _ in range(max(1, args.warmup // 3)):
        serve(arrivals, lps)
    clocks = ClockSampler(local)
    clocks.start()
    el, done, st = serve(arrivals, lps)
    el = max_over_ranks(el, dist, f"cuda:{local}")
    clk = clocks.stop()
    lat = [done[j][0] for j in range(len(lps))]
    opt = sum(1 for j in range(len(lps)) if done[j][1].termination == 0)
    st["terminations"] = term_hist(done[j][1].termination for j in range(len(lps)))
    orig_kkt = [done[j][1].rel_kkt_original for j in range(len(lps))
                if done[j][1].termination == 0]
    # the same requests at arrival rates the server keeps up with: the first
    # sweep_count requests, their arrival times rescaled to each rate
    sweep = []
    if args.sweep:
        k = min(args.sweep_count, len(lps))
        for lam in (float(v) for v in args.sweep.split(",")):
            arr_l = [a * args.rate / lam for a in arrivals[:k]]
            el_l, done_l, _ = serve(arr_l, lps[:k])
            lat_l = [done_l[j][0] for j in range(k)]
            sweep.append({"rate": lam, "requests": k, "offered_req_per_s": k / max(arr_l[-1], 1e-9),
                          "served_req_per_s": k / el_l,
                          "latency_p50_s": float(np.percentile(lat_l, 50)),
                          "latency_p99_s": float(np.percentile(lat_l, 99)),
                          "optimal": sum(1 for j in range(k) if done_l[j][1].termination == 0)})
    # comparator: each request solved singly, FP64, one after another
    t0 = time.perf_counter()
    single = []
    single_iters = []
    for lp in lps:
        ts = time.perf_counter()
        p = pkg.Problem(lp, dev)
        p.presolve(enable=presolve_rules(pkg, args))
        rs = p.solve(precision=pkg.LP_FP64)
        p.postsolve()
        p.close()
        single.append(time.perf_counter() - ts)
        single_iters.append(int(rs.iterations))
    t_single = time.perf_counter() - t0
    offered = len(lps) / max(reqs[-1].arrival_s, 1e-9)
    fifo = fifo_latencies([rq.arrival_s for rq in reqs], single)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on 8 requests spread over the size range: each presolved
        # and timed for a few PDHG iterations, extrapolated to the iteration
        # count the device's FP64 solve of that request needed
        idx = sorted(range(len(lps)), key=lambda j: lps[j].nnz)
        pick = [idx[int(q * (len(idx) - 1) / 7)] for q in range(8)] if len(idx) >= 8 else idx
        tot, spent = 0.0, 0.0
        for j in pick:
            est, _, sp = oracle_sample(lps[j], max(single_iters[j], 1), "c2", iters=2)
            tot += est
            spent += sp
        model, nproc = host_cpu()
        cpu = {"value": len(pick) / tot, "unit": "requests/s", "cores": 1, "kind": "oracle",
               "sample": f"EXTRAPOLATION: {len(pick)} requests spread over the size range "
                         f"(nnz {min(lps[j].nnz for j in pick)}-{max(lps[j].nnz for j in pick)}), "
                         "each: oracle presolve, set-up passes and 2 PDHG iterations timed, "
                         "extrapolated to the device FP64 solve's iteration count of that "
                         "request; served one after another",
               "host_cpu": model, "host_logical_cores": nproc,
               "cpu_seconds_spent": round(spent, 1)}
    line = {
        "metric": METRIC, "value": world * len(lps) / el, "unit": "requests/s", "n_gpus": world,
        "steps": 1, "warmup": max(1, args.warmup // 3), "ms_per_step": el * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == pkg.LP_FP64 else "f32 SpMV / f64 iterates", "data": "synthetic",
        "config": {"workload": desc, "requests": len(lps), "rate": args.rate,
                   "precision": args.precision, "sum_nnz": int(sum(lp.nnz for lp in lps)),
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2"},
        "offered_req_per_s": offered,
        "latency_p50_s": float(np.percentile(lat, 50)),
        "latency_p99_s": float(np.percentile(lat, 99)),
        "optimal": opt,
        "rel_kkt_original_after_postsolve_max": max(orig_kkt) if orig_kkt else None,
        "refinements": int(sum(done[j][1].refinements for j in range(len(lps)))),
        "rate_sweep": sweep,
        "single_fp64": {"requests_per_s": len(lps) / t_single,
                        "latency_p50_s": float(np.percentile(single, 50)),
                        "latency_p99_s": float(np.percentile(single, 99)),
                        "fifo_latency_p50_s": float(np.percentile(fifo, 50)),
                        "fifo_latency_p99_s": float(np.percentile(fifo, 99)),
                        "note": "each request presolved, solved and postsolved alone, in order; "
                                "latency = its own service time; fifo_latency = arrival to "
                                "completion if the same service times were served one at a "
                                "time in arrival order (the stream's arrival times)"},
        "server_stats": st,
        "e2e": {"value": world * len(lps) / el, "unit": "requests/s",
                "h2d_bytes_per_step": int(sum(lp.nnz * 24 for lp in lps)),
                "d2h_bytes_per_step": int(sum((2 * lp.n + lp.m) * 8 for lp in lps))},
        "cpu_baseline": cpu, "clocks": clk, "gpu_launches": st["launches"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("c4", "c5"):
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
