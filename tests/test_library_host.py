"""CPU-side checks of the C ABI library: it builds, loads without a GPU, and
exports every entry point that include/*.h declares; argument validation that
needs no device answers with the documented status codes."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2507_11512_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        names += re.findall(r"HPG_API\s+[\w\s\*]+?\b(hpg_\w+)\s*\(", text)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_2507_11512_gb300", "libhpgmxp.so"))
    for n in names:
        assert hasattr(raw, n), n


def test_binding_declares_every_symbol():
    from paper_2507_11512_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_status_strings(lib):
    assert lib.hpg_status_string(0) == b"HPG_OK"
    assert lib.hpg_status_string(-3) == b"HPG_ERR_NOT_CONVERGED"
    assert lib.hpg_status_string(-99) == b"HPG_ERR_UNKNOWN"


def test_host_side_validation_without_gpu(lib):
    from paper_2507_11512_gb300 import _lib
    out = ctypes.c_void_p()
    assert lib.hpg_setup_problem(0, 4, 4, None, ctypes.byref(out)) == _lib.HPG_ERR_INVALID
    assert out.value is None
    assert b"edge" in lib.hpg_last_error()
    assert lib.hpg_setup_problem(4, 4, 4, None, None) == _lib.HPG_ERR_INVALID
    p = _lib.StencilParams(2.0, None)
    assert lib.hpg_setup_problem(4, 4, 4, ctypes.byref(p), ctypes.byref(out)) == \
        _lib.HPG_ERR_INVALID
    assert lib.hpg_gmres_ir_solve(None, None, None, 1e-9, 30, 10, 1, 1, None, None) == \
        _lib.HPG_ERR_INVALID
    assert lib.hpg_spmv(None, 0, 1, None, None, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_mg_vcycle(None, 0, 1, None, None, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_mg_smooth(None, 0, 1, None, None, 1, 1, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_spmv_batch(None, 0, 8, None, None, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_mg_vcycle_batch(None, 0, 8, None, None, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_gmres_ir_solve_batch(None, 8, None, None, 1e-9, 30, 10, None, None) == \
        _lib.HPG_ERR_INVALID
    assert lib.hpg_batch_tune(None, 8, None) == _lib.HPG_ERR_INVALID
    out = ctypes.c_void_p()
    assert lib.hpg_batch_create(None, 0, 8, 30, ctypes.byref(out)) == _lib.HPG_ERR_INVALID
    assert lib.hpg_batch_solve(None, None, None, 1e-9, 10, None, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_batch_tune_solve(None, None, None, 1e-9, 10, None, None) == _lib.HPG_ERR_INVALID
    assert lib.hpg_batch_destroy(None) == _lib.HPG_OK
    assert lib.hpg_inject_stall(None, 0, 1) == _lib.HPG_ERR_INVALID
    assert lib.hpg_build_mg_hierarchy(None, 4, 1, 1) == _lib.HPG_ERR_INVALID
    assert lib.hpg_destroy(None) == _lib.HPG_OK
    assert lib.hpg_diag_scale_gradient(None, None, None, None, None) == _lib.HPG_ERR_INVALID
    cnt = ctypes.c_int()
    assert lib.hpg_profile_report(None, None, 0, ctypes.byref(cnt)) == _lib.HPG_ERR_INVALID


def test_build_is_idempotent():
    from paper_2507_11512_gb300 import build as b
    p1 = b.build()
    t1 = os.path.getmtime(p1)
    p2 = b.build()
    assert p1 == p2 and os.path.getmtime(p2) == t1
