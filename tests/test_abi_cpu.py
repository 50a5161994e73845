"""C ABI checks that need no GPU: the library loads, exports every entry point the header
declares, sizes workspaces, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

from paper_1903_12522_gb300 import cmcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(cmcg.LIB_PATH):
        from paper_1903_12522_gb300 import build

        build.build()
    return cmcg.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cmcg_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(cmcg.EXPORTED) <= set(names)


def test_checked_library_exports_the_same_symbols():
    # libcmcg_checked.so: the same sources with the kernels' compiled-in bounds checks
    if not os.path.exists(cmcg.LIB_CHECKED_PATH):
        from paper_1903_12522_gb300 import build

        build.build(checked=True)
    chk = C.CDLL(cmcg.LIB_CHECKED_PATH)
    for name in declared_functions():
        assert hasattr(chk, name), name


def test_workspace_size(lib):
    g = cmcg.make_grid((64, 48), 1 / 64)
    s64 = cmcg.cmcg_workspace_size(g, cmcg.make_options(cmcg.FP64))
    s32 = cmcg.cmcg_workspace_size(g, cmcg.make_options(cmcg.FP32))
    smx = cmcg.cmcg_workspace_size(g, cmcg.make_options(cmcg.MIXED))
    sio = cmcg.cmcg_workspace_size(g, cmcg.make_options(cmcg.FP64, flags=cmcg.FLAG_HOST_IO))
    npn = 65 * 49
    assert s64 > 20 * 8 * npn
    assert s64 < s32 < smx
    assert sio - s64 >= 16 * npn
    g3 = cmcg.make_grid((256, 256, 256), 1 / 256)
    assert cmcg.cmcg_workspace_size(g3, cmcg.make_options(cmcg.MIXED)) < 8 * 1024 ** 3


@pytest.mark.parametrize("bad", [
    dict(n=(1, 8)), dict(n=(8, 8), h=0.0), dict(n=(8, 8), order=3), dict(n=(8, 8, 8, 8)),
])
def test_workspace_size_rejects_invalid_grids(lib, bad):
    n = bad.get("n", (8, 8))
    g = cmcg.Grid()
    g.dim = len(n) if len(n) <= 3 else 4
    for a in range(min(3, len(n))):
        g.n[a] = n[a]
    g.h = bad.get("h", 0.125)
    g.order = bad.get("order", 2)
    assert cmcg.cmcg_workspace_size(g, cmcg.make_options()) == 0


def test_create_rejects_null_arguments_without_a_gpu(lib):
    g = cmcg.make_grid((8, 8), 0.125)
    o = cmcg.make_options()
    bc = cmcg.BC()
    h = C.c_void_p()
    code = lib.cmcg_create(C.byref(g), None, 1.0, C.byref(bc), C.byref(o), None, 0, None, C.byref(h))
    assert code == cmcg.ERR_INVALID_ARG and not h.value
    assert lib.cmcg_solve(None, None, None, 1e-6, None, None) == cmcg.ERR_INVALID_ARG
    assert lib.cmcg_solve_warm(None, None, None, 1e-6, None, None) == cmcg.ERR_INVALID_ARG
    assert lib.cmcg_wave_period(None, None, None, None, None, None, None) == cmcg.ERR_INVALID_ARG
    assert lib.cmcg_destroy(None) == cmcg.ERR_INVALID_ARG


def test_status_strings(lib):
    assert cmcg.cmcg_status_string(cmcg.OK) == "ok"
    assert "CFL" in cmcg.cmcg_status_string(cmcg.ERR_CFL)
    assert cmcg.cmcg_status_string(12345) == "unknown status"


def test_check_status_reports_no_checks_in_the_normal_build(lib):
    # the normal build compiles no bounds checks: zeros and ERR_UNSUPPORTED (the call only
    # synchronises the device, which a host without a GPU answers with an error code)
    c, si, ix = C.c_longlong(7), C.c_longlong(7), C.c_longlong(7)
    code = lib.cmcg_check_status(C.byref(c), C.byref(si), C.byref(ix))
    assert code in (cmcg.ERR_UNSUPPORTED, cmcg.ERR_CUDA)
    if code == cmcg.ERR_UNSUPPORTED:
        assert c.value == 0 and si.value == -1 and ix.value == 0


def test_missing_library_fails_loudly(tmp_path):
    saved = cmcg._lib
    cmcg._lib = None
    try:
        with pytest.raises(RuntimeError):
            cmcg.load(str(tmp_path / "libcmcg.so"))
    finally:
        cmcg._lib = saved
