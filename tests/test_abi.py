"""C-ABI checks that need no GPU: the library builds, loads, exports every
declared entry point, and rejects bad host arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1707_02162_gb300 import build as B
from paper_1707_02162_gb300 import redo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(redo_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return redo.load_library()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(redo.EXPORTS) <= declared


def test_host_validation_without_device(lib):
    out = ctypes.c_void_p()
    lo = (ctypes.c_double * 1)(-1.0)
    hi = (ctypes.c_double * 1)(1.0)
    dummy = ctypes.c_void_p(16)
    # N not a power of two / out of range: rejected before any CUDA call
    st = lib.redo_build_table(3, 1, 1e-6, dummy, dummy, ctypes.cast(lo, ctypes.c_void_p),
                              ctypes.cast(hi, ctypes.c_void_p), 64, 2, 0, None, ctypes.byref(out))
    assert st == 5 and b"N=3" in lib.redo_last_error()
    st = lib.redo_build_table(8, 0, 1e-6, dummy, dummy, ctypes.cast(lo, ctypes.c_void_p),
                              ctypes.cast(hi, ctypes.c_void_p), 64, 2, 0, None, ctypes.byref(out))
    assert st == 1
    st = lib.redo_build_table(8, 1, -1.0, dummy, dummy, ctypes.cast(lo, ctypes.c_void_p),
                              ctypes.cast(hi, ctypes.c_void_p), 64, 2, 0, None, ctypes.byref(out))
    assert st == 1
    st = lib.redo_build_table(8, 1, 1e-6, None, dummy, ctypes.cast(lo, ctypes.c_void_p),
                              ctypes.cast(hi, ctypes.c_void_p), 64, 2, 0, None, ctypes.byref(out))
    assert st == 1
    st = lib.redo_build_table(8, 1, 1e-6, dummy, dummy, ctypes.cast(hi, ctypes.c_void_p),
                              ctypes.cast(lo, ctypes.c_void_p), 64, 2, 0, None, ctypes.byref(out))
    assert st == 1 and b"lo < hi" in lib.redo_last_error()
    st = lib.redo_build_table(8, 1, 1e-6, dummy, dummy, ctypes.cast(lo, ctypes.c_void_p),
                              ctypes.cast(hi, ctypes.c_void_p), 4096, 3, 0, None, ctypes.byref(out))
    assert st == 1
    assert lib.redo_propagate(None, None, 1, 1, 0, 0, None, None, None, None, None, 0, None, None) == 1
    assert lib.redo_quantize(None, None, 1, 1, None, None, None) == 1
    assert lib.redo_table_free(None) == 0
    # per-pulse drift, amplitude/phase and time-split entry points: no table, bad sizes
    n = ctypes.c_size_t()
    assert lib.redo_propagate_drift(None, None, None, 1, 1, 0, 0, None, None, None, None, None, 0, None, None) == 1
    assert lib.redo_propagate_drift_workspace(None, 1, 1, 0, 0, ctypes.byref(n)) == 1
    assert lib.redo_fidelity_grad_drift(None, None, None, 1, 1, None, 0, 0, 0, None, None, None, 0, None, None) == 1
    assert lib.redo_fidelity_grad_drift_workspace(None, 1, 1, 0, 0, ctypes.byref(n)) == 1
    assert lib.redo_propagate_phase(None, None, None, 1, 1, 0, 0, None, None, None, None, None, 0, None, None) == 1
    assert lib.redo_fidelity_grad_phase(None, None, None, 1, 1, None, 0, 0, 0, None, None, None, None, 0, None,
                                        None) == 1
    assert lib.redo_batched_product(0, 1, dummy, 0, 0, dummy, 0, 0, dummy, None) == 1
    assert lib.redo_batched_product(8, -1, dummy, 0, 0, dummy, 0, 0, dummy, None) == 1
    assert lib.redo_batched_product(8, 0, dummy, 0, 0, dummy, 0, 0, dummy, None) == 0     # nothing to do


class _FakeTable:
    N = 4
    device = "cpu"


def test_propagation_wrappers_take_one_target():
    import numpy as np
    t = redo._single_target(_FakeTable(), np.eye(4))
    assert tuple(t.shape) == (4, 4)
    with pytest.raises(ValueError):
        redo._single_target(_FakeTable(), np.stack([np.eye(4)] * 2))


def test_build_flags_are_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
