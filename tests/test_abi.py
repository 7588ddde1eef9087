"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lslu.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2409_05239_gb300 import build as B
from paper_2409_05239_gb300 import lslu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            syms |= set(re.findall(r"\b(lslu_[a-z_0-9]+)\s*\(", src))
    return syms


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lslu.load()


def test_header_declares_entry_points():
    syms = declared_symbols()
    assert {"lslu_create", "lslu_solve", "lslu_destroy", "lslu_error_string"} <= syms
    assert syms == set(lslu.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (lslu_\w+)", out.stdout))
    assert declared_symbols() <= exported


def test_library_is_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", B.LIB], capture_output=True, text=True)
    assert "sm_103a" in out.stdout


def test_create_rejects_bad_arguments_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    h = ctypes.c_void_p()
    import numpy as np

    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([0, 5], dtype=np.int32)  # column 5 out of range for n = 2
    v = np.array([1.0, 2.0])
    st = lib.lslu_create(2, 2, 2, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 1, 10, 0, None,
                         ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG and not h.value
    assert b"column index" in lib.lslu_error_string(None)
    ci = np.array([0, 1], dtype=np.int32)
    rp_bad = np.array([0, 2, 1], dtype=np.int64)
    st = lib.lslu_create(2, 2, 1, rp_bad.ctypes.data, ci.ctypes.data, v.ctypes.data, 1, 10, 0,
                         None, ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG
    st = lib.lslu_create(2, 2, 2, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 1, 0, 0, None,
                         ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG
    vn = np.array([1.0, np.nan])
    st = lib.lslu_create(2, 2, 2, rp.ctypes.data, ci.ctypes.data, vn.ctypes.data, 1, 10, 0, None,
                         ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG and b"non-finite" in lib.lslu_error_string(None)


def test_create_batched_rejects_bad_arguments_without_gpu(lib):
    """Batch layout checks run before any CUDA call."""
    import numpy as np

    h = ctypes.c_void_p()
    ro = np.array([0, 1, 2], dtype=np.int64)
    co = np.array([0, 1, 2], dtype=np.int64)
    rp = np.array([0, 1, 2], dtype=np.int64)
    v = np.array([1.0, 2.0])

    def create(ro, co, ci, vt=1, nprob=2, v=v):
        return lib.lslu_create_batched(nprob, ro.ctypes.data, co.ctypes.data, rp.ctypes.data,
                                       ci.ctypes.data, v.ctypes.data, vt, 10, None,
                                       ctypes.byref(h))

    ok_ci = np.array([0, 1], dtype=np.int32)
    # FP64 values are not batched
    assert create(ro, co, ok_ci, vt=0) == lslu.ERR_INVALID_ARG and not h.value
    assert b"FP32 or BF16" in lib.lslu_error_string(None)
    # problem 1's row referencing problem 0's column
    assert create(ro, co, np.array([0, 0], dtype=np.int32)) == lslu.ERR_INVALID_ARG
    assert b"outside its problem" in lib.lslu_error_string(None)
    # an empty problem
    assert create(np.array([0, 2, 2], dtype=np.int64), co, ok_ci) == lslu.ERR_INVALID_ARG
    assert create(ro, co, ok_ci, nprob=0) == lslu.ERR_INVALID_ARG
    assert create(ro, co, ok_ci, v=np.array([1.0, np.inf])) == lslu.ERR_INVALID_ARG
    assert lib.lslu_solve_batched(None, None, 1, 2, 0.0, 0, None, None, None, None,
                                  None) == lslu.ERR_INVALID_ARG
    # shared-matrix handles: FP32/BF16 only, 1..16 right-hand sides
    rp2 = np.array([0, 1, 2], dtype=np.int64)
    st = lib.lslu_create_shared(2, 2, rp2.ctypes.data, ok_ci.ctypes.data, v.ctypes.data, 17, 1,
                                10, None, ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG and not h.value
    st = lib.lslu_create_shared(2, 2, rp2.ctypes.data, ok_ci.ctypes.data, v.ctypes.data, 2, 0,
                                10, None, ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG
    bad = np.array([0, 3], dtype=np.int32)
    st = lib.lslu_create_shared(2, 2, rp2.ctypes.data, bad.ctypes.data, v.ctypes.data, 2, 1,
                                10, None, ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG and b"column index" in lib.lslu_error_string(None)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lslu_solve(None, None, None, 1, 2, 0.0, 0, None, None, None, None, None,
                          None) == lslu.ERR_INVALID_ARG
    assert lib.lslu_last_launch_count(None) == 0
    lib.lslu_destroy(None)


def test_loop_control_rejects_bad_arguments_without_gpu(lib):
    assert lib.lslu_set_loop(None, 1, 0, 0, 0) == lslu.ERR_INVALID_ARG
    assert lib.lslu_loop_config(None, None, None, None) == lslu.ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        saved = lslu._lib
        lslu._lib = None
        try:
            lslu.load(str(tmp_path / "missing.so"))
        finally:
            lslu._lib = saved


def test_create_ordered_rejects_bad_orders_without_gpu(lib):
    """The renumbering checks of the three ordered creates run before any CUDA
    call: an order that is not a permutation, and a batch order that moves
    an index into another problem, are refused."""
    import numpy as np

    h = ctypes.c_void_p()
    rp = np.array([0, 1, 2], dtype=np.int64)
    ci = np.array([0, 1], dtype=np.int32)
    v = np.array([1.0, 2.0])
    ok = np.array([1, 0], dtype=np.int32)
    for ro, co in ((np.array([0, 0], np.int32), ok), (ok, np.array([0, 2], np.int32)),
                   (np.array([-1, 0], np.int32), None)):
        st = lib.lslu_create_ordered(2, 2, 2, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 1,
                                     10, ro.ctypes.data,
                                     None if co is None else co.ctypes.data, 0, None,
                                     ctypes.byref(h))
        assert st == lslu.ERR_INVALID_ARG and not h.value
        assert b"permutation" in lib.lslu_error_string(None)
    off = np.array([0, 1, 2], dtype=np.int64)
    swap = np.array([1, 0], dtype=np.int32)  # row 0 of problem 0 <-> row 0 of problem 1
    st = lib.lslu_create_batched_ordered(2, off.ctypes.data, off.ctypes.data, rp.ctypes.data,
                                         ci.ctypes.data, v.ctypes.data, 1, 10, swap.ctypes.data,
                                         None, None, ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG and b"onto themselves" in lib.lslu_error_string(None)
    st = lib.lslu_create_shared_ordered(2, 2, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 2,
                                        1, 10, None, np.array([1, 1], np.int32).ctypes.data,
                                        None, ctypes.byref(h))
    assert st == lslu.ERR_INVALID_ARG and b"permutation" in lib.lslu_error_string(None)


def test_stack_orders():
    """Per-problem orders become one global order of the batch: problem p's
    index i goes to off[p] + order_p[i]; None is the identity."""
    import numpy as np

    off = np.array([0, 3, 5, 9])
    g = lslu.stack_orders([(np.array([2, 0, 1]), None), (None, None),
                           (np.array([3, 2, 1, 0]), None)], 0, off)
    assert g.dtype == np.int32
    assert g.tolist() == [2, 0, 1, 3, 4, 8, 7, 6, 5]
    assert sorted(g.tolist()) == list(range(9))
