"""The C-ABI library: builds, loads, exports every declared symbol, and
rejects bad arguments on the host (no GPU needed for any of this)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2006_15234_gb300 import build, libpeps
    build.build_library()
    return libpeps.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "libpeps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(peps_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    from paper_2006_15234_gb300 import libpeps
    assert sorted(libpeps.EXPORTED_SYMBOLS) == names


def test_status_strings(lib):
    assert lib.peps_status_string(0) == b"PEPS_OK"
    assert lib.peps_status_string(5) == b"PEPS_ERR_WORKSPACE"
    assert b"sm_103a" in lib.peps_version()


def _net(lib_mod, nrow=2, ncol=2, d=2, D=2, dtype=1):
    bh = (C.c_int32 * (nrow * (ncol - 1)))(*([D] * (nrow * (ncol - 1))))
    bv = (C.c_int32 * ((nrow - 1) * ncol))(*([D] * ((nrow - 1) * ncol)))
    ptrs = (C.c_void_p * (nrow * ncol))(*([0x1000] * (nrow * ncol)))
    net = lib_mod.Network(nrow, ncol, d, dtype, C.cast(bh, C.POINTER(C.c_int32)),
                          C.cast(bv, C.POINTER(C.c_int32)), C.cast(ptrs, C.POINTER(C.c_void_p)))
    return net, (bh, bv, ptrs)


def test_plan_validation_errors(lib):
    from paper_2006_15234_gb300 import libpeps as L
    net, keep = _net(L)
    plan = C.c_void_p()
    ws = C.c_size_t()
    bad = L.make_opts(0, 4, 1, 1)
    assert lib.peps_contract_plan(C.byref(plan), C.byref(net), C.byref(net), C.byref(bad), 0,
                                  C.byref(ws)) == 1
    assert b"m must be" in lib.peps_last_error()
    good = L.make_opts(4, 4, 1, 1)
    # one-layer contraction requires d = 1
    assert lib.peps_contract_plan(C.byref(plan), C.byref(net), None, C.byref(good), 0, C.byref(ws)) == 2
    ok = lib.peps_contract_plan(C.byref(plan), C.byref(net), C.byref(net), C.byref(good), 0, C.byref(ws))
    assert ok == 0 and ws.value > 0
    # workspace NULL is refused before anything is enqueued
    assert lib.peps_contract_execute(plan, None, ws.value, None) == 5
    assert lib.peps_plan_destroy(plan) == 0


def test_einsumsvd_plan_sizes_and_rank(lib):
    from paper_2006_15234_gb300 import libpeps as L
    shapes = [(3, 4, 5, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2), (16, 9, 16, 16, 2, 3, 3, 3, 3, 3, 3, 3, 3)]
    arr = (L.EinsumsvdShape * 2)(*[L.EinsumsvdShape(*s) for s in shapes])
    plan = C.c_void_p()
    ws = C.c_size_t()
    opts = L.make_opts(16, 8, 2, 7)
    assert lib.peps_einsumsvd_plan(C.byref(plan), 1, 2, arr, None, C.byref(opts), C.byref(ws)) == 0
    k = C.c_int32()
    lib.peps_einsumsvd_rank(plan, 0, C.byref(k))
    assert k.value == min(16, 3 * 4, 2 * 2 * 3 * 2 * 2)
    lib.peps_einsumsvd_rank(plan, 1, C.byref(k))
    assert k.value == 16
    assert lib.peps_einsumsvd_rank(plan, 2, C.byref(k)) == 1
    lib.peps_plan_destroy(plan)
    # a zero dimension is a shape error
    bad = (L.EinsumsvdShape * 1)(L.EinsumsvdShape(0, 4, 5, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2))
    assert lib.peps_einsumsvd_plan(C.byref(plan), 1, 1, bad, None, C.byref(opts), C.byref(ws)) == 2


def test_workspace_query_matches_plan(lib):
    from paper_2006_15234_gb300 import libpeps as L
    net, keep = _net(L, 4, 4, 2, 3)
    opts = L.make_opts(6, 4, 2, 1)
    ws1 = C.c_size_t()
    assert lib.peps_boundary_workspace(C.byref(net), C.byref(net), C.byref(opts), C.byref(ws1)) == 0
    plan = C.c_void_p()
    ws2 = C.c_size_t()
    assert lib.peps_contract_plan(C.byref(plan), C.byref(net), C.byref(net), C.byref(opts), 0,
                                  C.byref(ws2)) == 0
    assert ws1.value == ws2.value
    lib.peps_plan_destroy(plan)
