"""The C ABI library loads and exports every function include/*.h declares,
and the Python binding marshals exactly those functions (CPU only: the
symbols are resolved, nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^[A-Za-z_][A-Za-z0-9_ ]*[ *]\s*(lp_[a-z0-9_]+)\s*\(", re.M)


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as f:
            src = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)  # drop comments
        names.update(DECL.findall(src))
    return names


def library():
    from paper_2604_23951_gb300 import capi

    if not os.path.exists(capi.LIB_PATH):
        pytest.skip("native library not built in this checkout")
    return capi, ctypes.CDLL(capi.LIB_PATH)


def test_headers_declare_the_boundary():
    names = declared()
    # the calls of the boundary: create from CSR, presolve, solve, postsolve,
    # batch submit / poll, and the server around them
    for core in ("lp_create", "lp_presolve", "lp_solve", "lp_postsolve", "lp_batch_submit",
                 "lp_batch_poll", "lp_server_create", "lp_server_destroy", "lp_destroy",
                 "lp_last_error"):
        assert core in names, core
    assert len(names) >= 30


def test_library_exports_every_declared_function():
    _, lib = library()
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_exactly_the_declared_functions():
    capi, _ = library()
    bound = {name for name, _, _ in capi.SIGNATURES}
    assert bound == declared(), (sorted(declared() - bound), sorted(bound - declared()))


def test_missing_library_fails_loudly(tmp_path):
    # no fallback: without the built library the package refuses to run
    from paper_2604_23951_gb300 import capi

    saved = capi._lib
    capi._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            capi.load(str(tmp_path / "absent.so"))
    finally:
        capi._lib = saved


class _NoDevice:
    """A device context with no allocator and no stream: enough for the
    checks lp_server_create makes before any device work."""

    def __init__(self, capi):
        self.ctx = capi.lp_device_ctx(capi.ALLOC_FN(), capi.FREE_FN(), None, None, 0)


@pytest.mark.parametrize("budget,opts,code", [
    (1 << 19, {}, -5),            # below 1 MiB: LP_ERR_BUDGET
    (2 << 20, {}, -5),            # cannot hold the slot tables: LP_ERR_BUDGET
    (1 << 30, {"polish": 1}, -1),  # the server keeps the default stopping test
    (1 << 30, {"eps_gap_rel": 1e-4}, -1),
])
def test_server_checks_come_before_device_work(budget, opts, code):
    capi, _ = library()
    import paper_2604_23951_gb300 as pkg

    with pytest.raises(pkg.LPError) as ei:
        pkg.Server(budget, _NoDevice(capi), **opts)
    assert ei.value.code == code
