"""ctypes binding of the C ABI in include/lp.h (argument marshalling only).

Every entry point keeps its C name.  Arrays are passed as numpy arrays (host
memory); device memory and the CUDA stream come from PyTorch through
:class:`TorchDevice`.  If the native library is missing the import fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgb300lp.so")

LP_OK, LP_PENDING = 0, 1
LP_ERR = {-1: "LP_ERR_INVALID", -2: "LP_ERR_OOM", -3: "LP_ERR_CUDA", -4: "LP_ERR_STATE",
          -5: "LP_ERR_BUDGET", -6: "LP_ERR_TIMEOUT"}
LP_OPTIMAL, LP_ITER_LIMIT, LP_TIME_LIMIT, LP_NUMERICAL, LP_INFEASIBLE, LP_UNBOUNDED, \
    LP_CANCELLED = range(7)
LP_FP64, LP_MIXED = 0, 1
LP_ENGINE_AUTO, LP_ENGINE_GRID, LP_ENGINE_CLUSTER = 0, 1, 2
LP_RULE_EMPTY_ROW, LP_RULE_EMPTY_COL, LP_RULE_FIXED_COL, LP_RULE_SINGLETON_ROW = 1, 2, 4, 8
LP_RULE_REDUNDANT_ROW, LP_RULE_DOUBLETON, LP_RULE_FREE_COL_SINGLETON = 16, 32, 64
LP_RULE_VARIABLE_LOCKS, LP_RULE_COL_SINGLETON_INEQ, LP_RULE_PARALLEL_ROWS = 128, 256, 512
LP_RULE_ALL = 1023
LP_RULE_PRIMAL_PROPAGATION = 1024  # opt-in, not in LP_RULE_ALL
LP_RULE_PARALLEL_COLS = 2048  # opt-in, not in LP_RULE_ALL
LP_RULE_DUAL_PROPAGATION = 4096  # opt-in, not in LP_RULE_ALL

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lp_device_ctx(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p),
                ("stream", C.c_void_p), ("device", C.c_int32)]


class lp_presolve_opts(C.Structure):
    _fields_ = [("max_rounds", C.c_int32), ("enable", C.c_int32)]


class lp_presolve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("rounds", C.c_int32), ("m", C.c_int32),
                ("n", C.c_int32), ("nnz", C.c_int64), ("m0", C.c_int32), ("n0", C.c_int32),
                ("nnz0", C.c_int64), ("counts", C.c_int64 * 16), ("seconds", C.c_double)]


class lp_solve_opts(C.Structure):
    _fields_ = [("eps_rel", C.c_double), ("max_iter", C.c_int64), ("time_limit_s", C.c_double),
                ("precision", C.c_int32), ("check_every", C.c_int32), ("rho", C.c_double),
                ("beta_suff", C.c_double), ("beta_nec", C.c_double), ("beta_art", C.c_double),
                ("theta", C.c_double), ("ruiz_iters", C.c_int32), ("pock_chambolle", C.c_int32),
                ("power_iters", C.c_int32), ("halpern", C.c_int32), ("restarts", C.c_int32),
                ("use_graph", C.c_int32), ("step_size", C.c_double),
                ("primal_weight", C.c_double), ("x_init", C.POINTER(C.c_double)),
                ("y_init", C.POINTER(C.c_double)), ("engine", C.c_int32),
                ("verbose", C.c_int32), ("infeas_every", C.c_int32),
                ("eps_infeas", C.c_double), ("primal_weight_clamp", C.c_double),
                ("refine_original", C.c_int32), ("tile_run_max", C.c_int32),
                ("tile_nnz", C.c_int32), ("eps_gap_rel", C.c_double), ("polish", C.c_int32),
                ("pad_polish_", C.c_int32), ("polish_fraction", C.c_double)]


class lp_result(C.Structure):
    _fields_ = [("termination", C.c_int32), ("restarts", C.c_int32), ("iterations", C.c_int64),
                ("rel_kkt", C.c_double), ("rel_p", C.c_double), ("rel_d", C.c_double),
                ("rel_gap", C.c_double), ("r_p", C.c_double), ("r_d", C.c_double),
                ("gap", C.c_double), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("eta", C.c_double), ("omega", C.c_double), ("t_setup_s", C.c_double),
                ("t_solve_s", C.c_double), ("t_total_s", C.c_double),
                ("kernel_launches", C.c_int64), ("fp32_iterations", C.c_int64),
                ("rel_kkt_original", C.c_double), ("refinements", C.c_int32),
                ("polish_attempts", C.c_int32), ("polished", C.c_int32), ("pad_", C.c_int32),
                ("polish_iterations", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# (name, restype, argtypes) of every exported function declared in include/lp.h
_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
SIGNATURES = [
    ("lp_solve_opts_default", None, [C.POINTER(lp_solve_opts)]),
    ("lp_presolve_opts_default", None, [C.POINTER(lp_presolve_opts)]),
    ("lp_last_error", C.c_char_p, []),
    ("lp_create", C.c_int, [C.c_int32, C.c_int32, C.c_int64, _I64, _I32, _D, _D, C.c_double,
                            _D, _D, _D, _D, C.POINTER(lp_device_ctx), _PP]),
    ("lp_presolve", C.c_int, [_P, C.POINTER(lp_presolve_opts), C.POINTER(lp_presolve_info)]),
    ("lp_upload", C.c_int, [_P]),
    ("lp_solve", C.c_int, [_P, C.POINTER(lp_solve_opts), C.POINTER(lp_result)]),
    ("lp_get_solution", C.c_int, [_P, _D, _D, _D]),
    ("lp_get_iterate", C.c_int, [_P, _D, _D]),
    ("lp_postsolve", C.c_int, [_P, _D, _D, _D]),
    ("lp_postsolve_from", C.c_int, [_P, _D, _D, _D, _D, _D, _D]),
    ("lp_get_dims", C.c_int, [_P, _I32, _I32, _I64, _I32, _I32]),
    ("lp_get_data", C.c_int, [_P, _I64, _I32, _D, _D, _D, _D, _D, _D, _D]),
    ("lp_host_rel_kkt", C.c_int, [_P, _D, _D, _D]),
    ("lp_profile_kernels", C.c_int, [_P, C.c_int32, _D]),
    ("lp_destroy", None, [_P]),
    ("lp_power_norm_static", C.c_int, [C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P, C.c_int32,
                                       _P, _D]),
    ("lp_server_create", C.c_int, [C.c_size_t, C.POINTER(lp_device_ctx),
                                   C.POINTER(lp_solve_opts), C.c_int32, _PP]),
    ("lp_batch_submit", C.c_int, [_P, _P, C.POINTER(C.c_uint64)]),
    ("lp_batch_poll", C.c_int, [_P, C.c_uint64, C.POINTER(lp_result), _D, _D]),
    ("lp_server_pump", C.c_int, [_P, C.c_int32]),
    ("lp_plan_rows", C.c_int, [C.c_int32, _I64, _I32, _I32, C.c_int32, _I32, _I32]),
    ("lp_plan_rows_shape", C.c_int, [C.c_int32, _I64, C.c_int32, C.c_int32, C.c_int32, _I32,
                                     _I32, C.c_int32, _I32, _I32, _I32, C.c_int32, _I32]),
    ("lp_get_tile_tuning", C.c_int, [_P, _D, C.c_int32, _I32]),
    ("lp_tile_cache_clear", None, []),
    ("lp_server_tune", C.c_int, [_P, C.c_int64, C.c_int32, C.c_double]),
    ("lp_batch_cancel", C.c_int, [_P, C.c_uint64]),
    ("lp_server_stats", C.c_int, [_P, _I64]),
    ("lp_server_graph_stats", C.c_int, [_P, _I64]),
    ("lp_server_tile_tuning", C.c_int, [_P, _D, C.c_int32, _I32]),
    ("lp_server_destroy", None, [_P]),
]

_lib = None


def load(path: str | None = None):
    """Load the native library (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"native library not built: {p} (run __graft_entry__.build())")
    lib = C.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{LP_ERR.get(code, code)}: {msg}")
        self.code = code


def check(rc):
    if rc < 0:
        raise LPError(rc, load().lp_last_error().decode())
    return rc


def dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def plan_rows(lengths):
    """Row order and warp tiles the device layout uses for rows of the given
    lengths (lp_plan_rows): (perm, tiles as an (ntiles, 2) int32 array of
    (first row, packed word), nlong)."""
    lib = load()
    L = np.ascontiguousarray(lengths, dtype=np.int64)
    rows = int(L.size)
    perm = np.zeros(max(rows, 1), dtype=np.int32)
    nt, nl = C.c_int32(), C.c_int32()
    cap = rows + 1
    tiles = np.zeros(2 * cap, dtype=np.int32)
    check(lib.lp_plan_rows(rows, L.ctypes.data_as(_I64), perm.ctypes.data_as(_I32),
                           tiles.ctypes.data_as(_I32), cap, C.byref(nt), C.byref(nl)))
    return perm[:rows], tiles[: 2 * nt.value].reshape(-1, 2), nl.value


def plan_rows_shape(lengths, run_max: int, tile_nnz: int, segmented: bool):
    """lp_plan_rows_shape: (perm, tiles (ntiles, 2), nlong, seg_base)."""
    lib = load()
    L = np.ascontiguousarray(lengths, dtype=np.int64)
    rows = int(L.size)
    perm = np.zeros(max(rows, 1), dtype=np.int32)
    nt, nl, ns = C.c_int32(), C.c_int32(), C.c_int32()
    seg_total = int(np.sum(-(-L // (32 * max(int(run_max), 1))))) if rows else 0
    cap = rows + seg_total + 1
    tiles = np.zeros(2 * cap, dtype=np.int32)
    sb = np.zeros(rows + 1, dtype=np.int32)
    check(lib.lp_plan_rows_shape(rows, L.ctypes.data_as(_I64), int(run_max), int(tile_nnz),
                                 1 if segmented else 0, perm.ctypes.data_as(_I32),
                                 tiles.ctypes.data_as(_I32), cap, C.byref(nt), C.byref(nl),
                                 sb.ctypes.data_as(_I32), rows + 1, C.byref(ns)))
    return (perm[:rows], tiles[: 2 * nt.value].reshape(-1, 2), nl.value,
            sb[: ns.value + 1])


def tile_cache_clear():
    load().lp_tile_cache_clear()


# --------------------------------------------------------------------------
# PyTorch-provided device memory and stream


class TorchDevice:
    """Device context backed by PyTorch: the caching allocator for device
    memory and a dedicated torch stream for the library's work."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        dev = device
        strm = self.stream

        def _alloc(nbytes, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
            except Exception:  # OOM is reported to the library as NULL
                return None

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc = ALLOC_FN(_alloc)
        self._free = FREE_FN(_free)
        self.ctx = lp_device_ctx(self._alloc, self._free, None, C.c_void_p(self.stream.cuda_stream),
                                 device)

    def synchronize(self):
        self.stream.synchronize()


def solve_opts(**kw) -> lp_solve_opts:
    o = lp_solve_opts()
    load().lp_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        if k in ("x_init", "y_init"):
            raise ValueError("pass warm starts to Problem.solve")
        setattr(o, k, v)
    return o


class Problem:
    """Owning wrapper of an lp_problem handle."""

    def __init__(self, lp, device: TorchDevice | None = None):
        lib = load()
        self.lib = lib
        self.device = device
        self.m0, self.n0 = int(lp.m), int(lp.n)
        rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
        va = _f64(lp.val)
        self._keep = None
        h = C.c_void_p()
        check(lib.lp_create(int(lp.m), int(lp.n), int(rp[-1]), rp.ctypes.data_as(_I64),
                            ci.ctypes.data_as(_I32), dptr(va), dptr(_f64(lp.c)),
                            float(getattr(lp, "obj_offset", 0.0)), dptr(_f64(lp.row_lo)),
                            dptr(_f64(lp.row_hi)), dptr(_f64(lp.col_lo)), dptr(_f64(lp.col_hi)),
                            C.byref(device.ctx) if device is not None else None, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            self.lib.lp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dims(self):
        m, n, m0, n0 = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        nnz = C.c_int64()
        check(self.lib.lp_get_dims(self.h, C.byref(m), C.byref(n), C.byref(nnz), C.byref(m0),
                                   C.byref(n0)))
        return m.value, n.value, nnz.value

    def presolve(self, max_rounds: int = 20, enable: int = LP_RULE_ALL) -> lp_presolve_info:
        o = lp_presolve_opts(max_rounds, enable)
        info = lp_presolve_info()
        check(self.lib.lp_presolve(self.h, C.byref(o), C.byref(info)))
        return info

    def upload(self):
        check(self.lib.lp_upload(self.h))

    def solve(self, x_init=None, y_init=None, **kw) -> lp_result:
        o = solve_opts(**kw)
        xi = _f64(x_init) if x_init is not None else None
        yi = _f64(y_init) if y_init is not None else None
        if xi is not None:
            o.x_init = dptr(xi)
        if yi is not None:
            o.y_init = dptr(yi)
        r = lp_result()
        check(self.lib.lp_solve(self.h, C.byref(o), C.byref(r)))
        return r

    def solution(self):
        m, n, _ = self.dims()
        x, y, z = np.zeros(n), np.zeros(m), np.zeros(n)
        check(self.lib.lp_get_solution(self.h, dptr(x), dptr(y), dptr(z)))
        return x, y, z

    def iterate(self):
        m, n, _ = self.dims()
        x, y = np.zeros(n), np.zeros(m)
        check(self.lib.lp_get_iterate(self.h, dptr(x), dptr(y)))
        return x, y

    def postsolve(self):
        x, y, z = np.zeros(self.n0), np.zeros(self.m0), np.zeros(self.n0)
        check(self.lib.lp_postsolve(self.h, dptr(x), dptr(y), dptr(z)))
        return x, y, z

    def postsolve_from(self, xr, yr, zr=None):
        x, y, z = np.zeros(self.n0), np.zeros(self.m0), np.zeros(self.n0)
        xr, yr = _f64(xr), _f64(yr)
        zr = _f64(zr) if zr is not None else None
        check(self.lib.lp_postsolve_from(self.h, dptr(xr), dptr(yr), dptr(zr), dptr(x),
                                         dptr(y), dptr(z)))
        return x, y, z

    def data(self):
        """The current (after presolve: reduced) LP as a plain namespace."""
        m, n, nnz = self.dims()
        rp = np.zeros(m + 1, np.int64)
        ci = np.zeros(nnz, np.int32)
        va, c = np.zeros(nnz), np.zeros(n)
        lo, hi, lx, ux = np.zeros(m), np.zeros(m), np.zeros(n), np.zeros(n)
        off = C.c_double()
        check(self.lib.lp_get_data(self.h, rp.ctypes.data_as(_I64), ci.ctypes.data_as(_I32),
                                   dptr(va), dptr(c), C.byref(off), dptr(lo), dptr(hi),
                                   dptr(lx), dptr(ux)))

        class _NS:
            pass

        ns = _NS()
        ns.m, ns.n, ns.row_ptr, ns.col_idx, ns.val, ns.c = m, n, rp, ci, va, c
        ns.obj_offset, ns.row_lo, ns.row_hi, ns.col_lo, ns.col_hi = off.value, lo, hi, lx, ux
        return ns

    def profile_kernels(self, reps: int = 20):
        out = np.zeros(8)
        check(self.lib.lp_profile_kernels(self.h, int(reps), dptr(out)))
        keys = ("primal_ms", "dual_ms", "primal_bytes", "dual_bytes", "kkt_rows_ms",
                "kkt_cols_ms", "kkt_rows_bytes", "kkt_cols_bytes")
        return dict(zip(keys, out))

    def tile_tuning(self):
        """The grid engine's tile shapes of the last solve (lp_get_tile_tuning):
        {"A": index, "T": index, "measured": bool, "shapes": [(run_max,
        tile_nnz)], "ms_A": [...], "ms_T": [...]}"""
        out = np.zeros(128)
        k = C.c_int32()
        check(self.lib.lp_get_tile_tuning(self.h, dptr(out), 128, C.byref(k)))
        nc = (k.value - 3) // 4
        q = out[3:3 + 4 * nc].reshape(nc, 4)
        return {"A": int(out[0]), "T": int(out[1]), "measured": bool(out[2]),
                "shapes": [(int(a), int(b)) for a, b in q[:, :2]],
                "ms_A": q[:, 2].tolist(), "ms_T": q[:, 3].tolist()}

    def rel_kkt(self, x, y):
        out = np.zeros(6)
        check(self.lib.lp_host_rel_kkt(self.h, dptr(_f64(x)), dptr(_f64(y)), dptr(out)))
        return dict(zip(("rel_kkt", "rel_p", "rel_d", "rel_gap", "p", "d"), out))


class Server:
    """Continuous-batching server (lp_server_*): problems are queued with
    submit(), admitted into the device arena as memory frees up, and solved
    by the batched kernel; poll() returns the result when it is done."""

    def __init__(self, budget_bytes: int, device: TorchDevice, worker: bool = False, **opts):
        self.lib = load()
        self.device = device
        o = solve_opts(**opts)
        h = C.c_void_p()
        check(self.lib.lp_server_create(int(budget_bytes), C.byref(device.ctx), C.byref(o),
                                        1 if worker else 0, C.byref(h)))
        self.h = h
        self._problems = {}

    def submit(self, problem: "Problem") -> int:
        t = C.c_uint64()
        check(self.lib.lp_batch_submit(self.h, problem.h, C.byref(t)))
        self._problems[t.value] = problem
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (lp_result, x, y) for the problem's current LP."""
        p = self._problems[ticket]
        m, n, _ = p.dims()
        x, y = np.zeros(n), np.zeros(m)
        r = lp_result()
        rc = check(self.lib.lp_batch_poll(self.h, C.c_uint64(ticket), C.byref(r), dptr(x),
                                          dptr(y)))
        if rc == LP_PENDING:
            return None
        del self._problems[ticket]
        return r, x, y

    def pump(self, periods: int = 1) -> int:
        return check(self.lib.lp_server_pump(self.h, int(periods)))

    def tune(self, solo_nnz: int = 0, solo_max: int = -1, launch_ms: float = 0.0):
        """Scheduler settings (lp_server_tune); non-positive values keep the default."""
        check(self.lib.lp_server_tune(self.h, int(solo_nnz), int(solo_max), float(launch_ms)))

    def cancel(self, ticket: int):
        check(self.lib.lp_batch_cancel(self.h, C.c_uint64(ticket)))

    def stats(self):
        out = np.zeros(12, dtype=np.int64)
        check(self.lib.lp_server_stats(self.h, out.ctypes.data_as(_I64)))
        keys = ("admitted", "finished", "periods", "peak_resident_bytes", "launches",
                "queued", "shape_b0", "shape_b1", "shape_b2", "shape_b3", "host_launch_ns",
                "device_launch_ns")
        return dict(zip(keys, (int(v) for v in out)))

    def graph_stats(self):
        """lp_server_graph_stats: bucket launches replayed from a CUDA graph
        and graphs instantiated."""
        out = np.zeros(2, dtype=np.int64)
        check(self.lib.lp_server_graph_stats(self.h, out.ctypes.data_as(_I64)))
        return {"graph_launches": int(out[0]), "graphs": int(out[1])}

    def tile_tuning(self):
        """lp_server_tile_tuning: per request class, the chosen tile shape (or
        -1), mean ns per nonzero-iteration and samples of each shape."""
        cnt = C.c_int32()
        cap = 256
        out = np.zeros(15 * cap)
        check(self.lib.lp_server_tile_tuning(self.h, out.ctypes.data_as(_D), cap,
                                             C.byref(cnt)))
        rows = out[: 15 * cnt.value].reshape(-1, 15)
        return [{"m_bucket": int(r[0]), "len_bucket": int(r[1]), "chosen": int(r[2]),
                 "mean_ns": [float(v) for v in r[3:9]], "samples": [int(v) for v in r[9:15]]}
                for r in rows]

    def run_all(self, tickets, max_periods: int = 1_000_000):
        """Drive the device loop (non-worker servers) until every ticket is done."""
        results = {}
        pending = list(tickets)
        for _ in range(max_periods):
            left = []
            for t in pending:
                got = self.poll(t)
                if got is None:
                    left.append(t)
                else:
                    results[t] = got
            pending = left
            if not pending:
                break
            self.pump(1)
        return results

    def close(self):
        if self.h:
            self.lib.lp_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
