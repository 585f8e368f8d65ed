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
    assert lib.redo_fidelity_grad_drift(None, None, None, 1, 1, None, 0, 0, 0, 0, None, None, None, 0, None,
                                        None) == 1
    assert lib.redo_fidelity_grad(None, None, 1, 1, None, 0, 0, 0, 0, None, None, None, 0, None, None) == 1
    assert lib.redo_grape_lbfgs_workspace(None, 1, 1, 8, ctypes.byref(n)) == 1
    assert lib.redo_grape_lbfgs_step(None, None, None, None, 1, 1, 8, 1, 0.05, 1e-4, None, 0, None, None, None) == 1
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


def test_plan_through_the_c_abi_matches_the_printed_cost_model(lib):
    # Section II's worked example and Section IV's freezing grain, as printed
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "worked_examples.json")))
    for key in ("coarse_grain_example", "freezing_grain"):
        e = g[key]
        assert redo.redo_plan(e["omega_max"], e["eps"], e["base"]) == (e["l"], e["m"], e["p"], e["s"])
    # the covered range: b^(m+1) > omega_max >= b^m, and b^l <= eps < b^(l+1)
    for om, eps, b in [(1e3, 1.0, 2), (65535.0, 1.0, 16), (2 * 3.141592653589793 * 1e4, 30.7, 64), (0.5, 0.01, 10)]:
        l, m, p, s = redo.redo_plan(om, eps, b)
        assert b ** (m + 1) > om >= b ** m and b ** l <= eps * (1 + 1e-12) < b ** (l + 1)
        assert p == m - l and s == (b - 1) * (m - l + 1)
    with pytest.raises(redo.RedoError):
        redo.redo_plan(-1.0, 1.0, 64)
    with pytest.raises(redo.RedoError):
        redo.redo_plan(10.0, 1.0, 1)


def test_new_entry_points_validate_without_device(lib):
    n = ctypes.c_size_t()
    dummy = ctypes.c_void_p(16)
    assert lib.redo_propagate_steps(None, None, 1, 1, 0, None, None, 0, None, None) == 1
    assert lib.redo_propagate_steps_workspace(None, 1, 1, 0, ctypes.byref(n)) == 1
    assert lib.redo_reunitarize(3, 1, 0, dummy, dummy, 1, None) == 5          # N not a power of two
    assert lib.redo_reunitarize(128, 1, 0, dummy, dummy, 1, None) == 5        # beyond the shared-memory kernel
    assert lib.redo_reunitarize(8, 1, 4, dummy, dummy, 1, None) == 5          # FP64 / FP32 arithmetic only
    assert lib.redo_reunitarize(8, -1, 0, dummy, dummy, 1, None) == 1
    assert lib.redo_reunitarize(8, 0, 0, None, None, 1, None) == 0            # nothing to do


def test_mlp_sizes_through_the_binding(lib):
    # the warm-start network 23 -> 3 x 512 GELU -> 5000: params = sum of W (out x in) and b (out)
    sizes = [23, 512, 512, 512, 5000]
    want = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    assert want == 3_102_600                               # the 3.10 M parameters of the warm-start network
    for batch in (0, 1, 256):
        p, a, w = redo.redo_mlp_sizes(sizes, batch)
        assert p == want
        # z and h of every layer for `batch` samples come first in acts; two gradient buffers of
        # the widest layer in work
        assert a >= 2 * batch * sum(sizes[1:])
        assert w >= 2 * batch * max(sizes)
    with pytest.raises(redo.RedoError):
        redo.redo_mlp_sizes([23], 4)                      # no layer
    with pytest.raises(redo.RedoError):
        redo.redo_mlp_sizes([23, 0, 5], 4)                # empty layer
    with pytest.raises(redo.RedoError):
        redo.redo_mlp_sizes([23, 5], -1)                  # negative batch


def test_binding_rejects_host_tensors():
    import torch
    with pytest.raises(ValueError, match="device tensor"):
        redo._ptr(torch.zeros(4))
    assert redo._ptr(None) is None


_HOST_FUZZ = r'''
import ctypes, itertools, math, sys
sys.path.insert(0, sys.argv[1])
from paper_1707_02162_gb300 import redo
L = redo.load_library()
vals = [0.0, -1.0, 1e-320, 1e-300, 1e-12, 0.5, 1.0, 64.0, 2.6e5, 1e300, math.inf, -math.inf, math.nan]
bases = [-5, 0, 1, 2, 3, 64, 100, 2 ** 31 - 1]
out = [ctypes.c_int32() for _ in range(3)] + [ctypes.c_int64()]
seen = set()
for om, eps, b in itertools.product(vals, vals, bases):
    st = L.redo_plan(om, eps, b, *[ctypes.byref(o) for o in out])
    seen.add(st)
    if st == 0:
        l, m, p, s = (o.value for o in out)
        assert p == m - l >= -1 and s == (b - 1) * (m - l + 1), (om, eps, b, l, m, p, s)
        assert b ** l <= eps * (1 + 1e-12) < b ** (l + 1) * (1 + 1e-9) or eps < 1e-300
    else:
        assert st == 1, st
for sizes in ([23], [23, 512, 5000], [1] * 34, [4, 1 << 20, 3], [0, 2], [5, -1, 2]):
    arr = (ctypes.c_int32 * len(sizes))(*sizes)
    for batch in (-1, 0, 1, 1 << 20):
        p, a, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        st = L.redo_mlp_sizes(len(sizes) - 1, ctypes.cast(arr, ctypes.c_void_p), batch,
                              ctypes.byref(p), ctypes.byref(a), ctypes.byref(w))
        assert st in (0, 1), st
        if st == 0:
            assert p.value > 0 and a.value >= 0 and w.value >= 0
print("ok", sorted(seen))
'''


def test_host_only_entry_points_survive_edge_inputs(lib):
    # run in a child process: a crash on some input fails this test instead of the whole session
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _HOST_FUZZ, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.startswith("ok")


@pytest.fixture
def fake_table():
    """A handle whose (N, K) = (4, 3) sits in the binding's cache; no library table behind it."""
    h = 987654321
    redo._TABLE_NK[h] = (4, 3)
    yield h
    redo._TABLE_NK.pop(h, None)


def _past_checks(fn, *a, **kw):
    # correct sizes reach the device check, which host tensors then fail
    with pytest.raises(ValueError, match="device tensor expected"):
        fn(*a, **kw)


def test_binding_checks_sizes_against_the_table(fake_table):
    import torch
    h, B, M, N, K = fake_table, 2, 5, 4, 3
    u = torch.zeros((B, M, K), dtype=torch.float64)
    q = torch.zeros((B, M, K), dtype=torch.int32)
    _past_checks(redo.redo_quantize, h, u, q)
    with pytest.raises(ValueError, match="elements expected"):
        redo.redo_quantize(h, torch.zeros((B, M, K + 1), dtype=torch.float64), q)
    with pytest.raises(ValueError, match="int32 expected"):
        redo.redo_quantize(h, u, q.to(torch.int64))
    with pytest.raises(ValueError, match="float64 expected"):
        redo.redo_quantize(h, u.float(), q)
    ws = torch.zeros(256, dtype=torch.uint8)
    U = torch.zeros((B, N, N), dtype=torch.complex128)
    _past_checks(redo.redo_propagate, h, q, "fp64", U, None, None, None, ws)
    with pytest.raises(ValueError, match="elements expected"):
        redo.redo_propagate(h, q[:, :, :2].contiguous(), "fp64", U, None, None, None, ws)
    with pytest.raises(ValueError, match="U_out"):
        redo.redo_propagate(h, q, "fp64", U[:1], None, None, None, ws)
    with pytest.raises(ValueError, match="F_out"):
        redo.redo_propagate(h, q, "fp64", U, torch.zeros((N, N), dtype=torch.complex128),
                            torch.zeros(1, dtype=torch.float64), None, ws)
    g = torch.zeros((B, M, K), dtype=torch.float64)
    T = torch.zeros((N, N), dtype=torch.complex128)
    F = torch.zeros(B, dtype=torch.float64)
    _past_checks(redo.redo_fidelity_grad, h, q, T, "fp64", 0, F, g, ws)
    with pytest.raises(ValueError, match="grad"):
        redo.redo_fidelity_grad(h, q, T, "fp64", 0, F, g[:, :2], ws)
    with pytest.raises(ValueError, match="U_target"):
        redo.redo_fidelity_grad(h, q, torch.zeros((1, N, N), dtype=torch.complex128), "fp64", 0, F, g, ws)
    _past_checks(redo.redo_grape_step, h, u, g, 0.1)
    with pytest.raises(ValueError, match="step_scale"):
        redo.redo_grape_step(h, u, g, 0.1, torch.ones(1, dtype=torch.float64))
    _past_checks(redo.redo_grape_adam_step, h, u, g, torch.zeros_like(u), torch.zeros_like(u), 1, 0.01)
    with pytest.raises(ValueError, match="elements expected"):
        redo.redo_grape_adam_step(h, torch.zeros((B, M, K + 2), dtype=torch.float64), g, g, g, 1, 0.01)
    psi = torch.zeros(N, dtype=torch.complex128)
    _past_checks(redo.redo_simulate, h, q, "fp64", 0, psi, torch.zeros(N, dtype=torch.float64),
                 torch.zeros((B, M + 1), dtype=torch.float64), None, None)
    with pytest.raises(ValueError, match="expect"):
        redo.redo_simulate(h, q, "fp64", 0, psi, torch.zeros(N, dtype=torch.float64),
                           torch.zeros((B, M), dtype=torch.float64), None, None)
    # an empty pulse (M = 0) of a K = 1 table may drop its last axis
    redo._TABLE_NK[h] = (4, 1)
    _past_checks(redo.redo_quantize, h, torch.zeros((3, 7), dtype=torch.float64), torch.zeros((3, 7), dtype=torch.int32))
    _past_checks(redo.redo_propagate, h, torch.zeros((3, 0, 1), dtype=torch.int32), "fp64",
                 torch.zeros((3, N, N), dtype=torch.complex128), None, None, None, ws)


def test_binding_checks_products_reunitarisation_and_mlp_arrays(lib):
    import torch
    N = 4
    A = torch.zeros((3, N, N), dtype=torch.complex128)
    _past_checks(redo.redo_batched_product, A, torch.zeros((N, N), dtype=torch.complex128))
    with pytest.raises(ValueError, match="batches differ"):
        redo.redo_batched_product(A, torch.zeros((2, N, N), dtype=torch.complex128))
    with pytest.raises(ValueError, match="complex128"):
        redo.redo_batched_product(A, torch.zeros((3, N, N + 1), dtype=torch.complex128))
    with pytest.raises(ValueError, match="complex128"):
        redo.redo_batched_product(A, torch.zeros((3, N, N), dtype=torch.complex64))
    with pytest.raises(ValueError, match="out"):
        redo.redo_batched_product(A, A, out=torch.zeros((2, N, N), dtype=torch.complex128))
    _past_checks(redo.redo_reunitarize, A, torch.empty_like(A))
    with pytest.raises(ValueError, match="P_in"):
        redo.redo_reunitarize(A.to(torch.complex64), torch.empty_like(A))
    with pytest.raises(ValueError, match="U_out"):
        redo.redo_reunitarize(A, torch.empty((2, N, N), dtype=torch.complex128))
    sizes, batch = [5, 7, 3], 4
    p, a, w = redo.redo_mlp_sizes(sizes, batch)
    params = torch.zeros(p, dtype=torch.float32)
    x = torch.zeros((batch, 5), dtype=torch.float32)
    acts = torch.zeros(a, dtype=torch.float32)
    y = torch.zeros((batch, 3), dtype=torch.float32)
    _past_checks(redo.redo_mlp_forward, sizes, params, x, acts, y)
    with pytest.raises(ValueError, match="params"):
        redo.redo_mlp_forward(sizes, params[:-1], x, acts, y)
    with pytest.raises(ValueError, match="x"):
        redo.redo_mlp_forward(sizes, params, torch.zeros((batch, 6), dtype=torch.float32), acts, y)
    with pytest.raises(ValueError, match="acts"):
        redo.redo_mlp_forward(sizes, params, x, acts[:-1], y)
    work, grads = torch.zeros(w, dtype=torch.float32), torch.zeros(p, dtype=torch.float32)
    _past_checks(redo.redo_mlp_backward, sizes, params, x, acts, y, grads, None, work)
    with pytest.raises(ValueError, match="work"):
        redo.redo_mlp_backward(sizes, params, x, acts, y, grads, None, work[:-1])
    _past_checks(redo.redo_mlp_adam, params, grads, grads.clone(), grads.clone(), 1, 1e-3)
    with pytest.raises(ValueError, match="float32"):
        redo.redo_mlp_adam(params.double(), grads, grads, grads, 1, 1e-3)


def test_binding_checks_table_build_inputs():
    import torch
    N, K = 4, 2
    H0 = torch.zeros((N, N), dtype=torch.complex128)
    Hk = torch.zeros((K, N, N), dtype=torch.complex128)
    with pytest.raises(ValueError, match="device tensor expected"):
        redo.redo_build_table(H0, Hk, 1e-6, [-1.0, -1.0], [1.0, 1.0], 64, 2)
    with pytest.raises(ValueError, match="one per control term"):
        redo.redo_build_table(H0, Hk, 1e-6, [-1.0], [1.0], 64, 2)
    with pytest.raises(ValueError, match=r"Hk \[K\]\[N\]\[N\]"):
        redo.redo_build_table(H0, torch.zeros((K, N, N + 1), dtype=torch.complex128), 1e-6, [-1.0] * 2, [1.0] * 2, 64, 2)
    with pytest.raises(ValueError, match="complex128"):
        redo.redo_build_table(H0.to(torch.complex64), Hk, 1e-6, [-1.0] * 2, [1.0] * 2, 64, 2)


def test_binding_checks_phase_axes(fake_table):
    import numpy as np
    with pytest.raises(ValueError, match="sz"):
        redo.redo_table_set_phase_axes(fake_table, np.zeros((3, 3)))
