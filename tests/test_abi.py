"""The C-ABI library loads and exports every function include/gj.h declares;
argument checks fail with GJ_ERR_ARG before any device work (runs without a GPU)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "gj.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gj_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2112_15562_gb300 import _lib

    return _lib.load()


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_argument_errors_without_device_work(lib):
    from paper_2112_15562_gb300 import _lib as L

    out = ct.c_void_p()
    assert lib.gj_bttb_setup(None, 1, None, 0, 0, 0, None, ct.byref(out)) == -1
    assert b"grid" in lib.gj_last_error()
    z = (ct.c_double * 3)(0.0, 10.0, 20.0)
    g = L.Grid(4, 4, 4, 4, 2, 10.0, 10.0, ct.cast(z, ct.POINTER(ct.c_double)), 0.0, 0, 0)
    assert lib.gj_bttb_setup(ct.byref(g), 7, None, 0, 0, 0, None, ct.byref(out)) == -1
    assert lib.gj_bttb_setup(ct.byref(g), 2, None, 0, 0, 0, None, ct.byref(out)) == -1  # magnetic without gj_mag
    assert lib.gj_bttb_setup(ct.byref(g), 1, None, 0, 5, 5, None, ct.byref(out)) == -1  # padded size too small
    g.nz = 0
    assert lib.gj_bttb_setup(ct.byref(g), 1, None, 0, 0, 0, None, ct.byref(out)) == -1
    assert lib.gj_g_forward(None, None, None, None) == -1
    assert lib.gj_g_adjoint(None, None, None, None) == -1
    assert lib.gj_gramian_value_grad(0, 0, None, None, None, None, None, None) == -1
    assert lib.gj_rrcg_create(None, None, None, None, None, None, None, None, None, None, ct.byref(out)) == -1
    assert lib.gj_rrcg_iterate(None, 1, 0, None) == -1
    assert lib.gj_op_info(None, None) == -1
    assert lib.gj_op_status(None, 1, None) == -1
    assert lib.gj_selftest_bounded_wait(-1, None) == -1
    assert lib.gj_selftest_bounded_wait(10**11, None) == -1
    lib.gj_op_destroy(None)
    lib.gj_rrcg_destroy(None)
    assert lib.gj_version().startswith(b"gj")
