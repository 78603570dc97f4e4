"""The C-ABI library loads without a GPU and exports every function include/ilu2l.h
declares; the host-only entry points behave as documented. No compute calls here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    hdr = open(os.path.join(ROOT, "include", "ilu2l.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       hdr, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "for", "while")))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as ilu
    return ilu.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("ilu_setup", "ilu_apply", "gmres_solve", "ilu_free", "ilu_status_str",
                 "ilu_opts_default"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_defaults(lib):
    import paper_2303_08881_gb300 as ilu
    assert ilu.status_str(0) == "ok"
    assert ilu.status_str(2) == "malformed CSR matrix"
    o = ilu.ilu_opts()
    lib.ilu_opts_default(C.byref(o))
    assert (o.variant, o.factor_B, o.factor_S, o.inner_iters, o.pc_precision) == (1, 0, 1, 3, 1)
    assert o.pivot_eps == 1e-8 and o.use_graphs == 1


def test_setup_rejects_bad_arguments_without_touching_the_gpu(lib):
    """argument and CSR checks run on the host before any device call"""
    import numpy as np
    import paper_2303_08881_gb300 as ilu
    h = C.c_void_p()
    assert lib.ilu_setup(None, None, 1, None, C.byref(h)) == ilu.ILU_ERR_ARG
    rp = np.array([0, 2, 3], np.int32)
    ci = np.array([1, 0, 1], np.int32)          # row 0 unsorted
    v = np.ones(3)
    part = np.zeros(2, np.int32)
    A = ilu.ilu_csr(2, 3, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    o = ilu.ilu_opts()
    lib.ilu_opts_default(C.byref(o))
    assert lib.ilu_setup(C.byref(A), part.ctypes.data_as(C.c_void_p), 1, C.byref(o), C.byref(h)) == ilu.ILU_ERR_CSR
    ci2 = np.array([0, 1, 0], np.int32)          # row 1 misses its diagonal
    A2 = ilu.ilu_csr(2, 3, rp.ctypes.data, ci2.ctypes.data, v.ctypes.data)
    assert lib.ilu_setup(C.byref(A2), part.ctypes.data_as(C.c_void_p), 1, C.byref(o), C.byref(h)) == ilu.ILU_ERR_CSR
    ci3 = np.array([0, 1, 1], np.int32)
    A3 = ilu.ilu_csr(2, 3, rp.ctypes.data, ci3.ctypes.data, v.ctypes.data)
    bad = np.array([0, 5], np.int32)             # part out of range
    assert lib.ilu_setup(C.byref(A3), bad.ctypes.data_as(C.c_void_p), 2, C.byref(o), C.byref(h)) == ilu.ILU_ERR_ARG
    o.inner_iters = 0
    assert lib.ilu_setup(C.byref(A3), part.ctypes.data_as(C.c_void_p), 1, C.byref(o), C.byref(h)) == ilu.ILU_ERR_ARG
    assert not h.value
    assert lib.ilu_free(None) == 0
