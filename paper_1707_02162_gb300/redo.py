"""Thin ctypes binding of libredo (argument marshalling only).

Every function here forwards to the C entry point of the same name declared in
``include/redo.h``; torch is used only to own device memory and to name the
current CUDA stream.  There is no CPU fallback: if ``libredo.so`` is missing or
no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libredo.so")

REDO_OK = 0
REDO_FP64, REDO_FP32, REDO_FP16X3 = 0, 1, 4
PRECISIONS = {"fp64": REDO_FP64, "fp32": REDO_FP32, "fp16x3": REDO_FP16X3}
REDO_TABLE_FP32, REDO_TABLE_FP16X3, REDO_TABLE_LEVELS, REDO_TABLE_STRANG = 0x1, 0x2, 0x4, 0x8
STATUS_WORDS = 4
STATUS_NONFINITE, STATUS_SATURATED, STATUS_TIMEOUT, STATUS_BADINDEX = range(4)

EXPORTS = [
    "redo_build_table", "redo_table_free", "redo_table_info", "redo_table_copy", "redo_quantize",
    "redo_propagate", "redo_propagate_workspace", "redo_last_error", "redo_profile_enable",
    "redo_profile_read", "redo_propagate_noalloc", "redo_fidelity_grad", "redo_fidelity_grad_workspace",
    "redo_grape_step", "redo_simulate", "redo_simulate_workspace", "redo_mlp_sizes", "redo_mlp_forward",
    "redo_mlp_backward", "redo_mlp_adam", "redo_grape_adam_step", "redo_expect_diag",
    "redo_state_grad", "redo_state_grad_workspace", "redo_table_set_phase_axes", "redo_propagate_phase",
    "redo_propagate_phase_workspace", "redo_batched_product", "redo_fidelity_grad_phase",
    "redo_fidelity_grad_phase_workspace", "redo_propagate_drift", "redo_propagate_drift_workspace",
    "redo_fidelity_grad_drift", "redo_fidelity_grad_drift_workspace", "redo_propagate_steps",
    "redo_propagate_steps_workspace", "redo_reunitarize", "redo_plan", "redo_grape_lbfgs_workspace",
    "redo_grape_lbfgs_step",
]
PROFILE_PHASES = 11
PHASE_NAMES = ["quantize", "table", "chain_segments", "chain_combine", "finalize", "chain_tc", "reunitarize",
               "gradient", "grad_forward_sweep", "grad_scans", "grad_reverse_sweep"]


class RedoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libredo status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libredo.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_1707_02162_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
    L.redo_build_table.argtypes = [i32, i32, dbl, vp, vp, vp, vp, i32, i32, u32, vp, ctypes.POINTER(vp)]
    L.redo_table_free.argtypes = [vp]
    L.redo_table_info.argtypes = [vp] + [ctypes.POINTER(i32)] * 4 + [ctypes.POINTER(i64)] * 2
    L.redo_table_copy.argtypes = [vp, vp, vp, vp]
    L.redo_quantize.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    L.redo_propagate.argtypes = [vp, vp, i64, i64, i32, i32, vp, vp, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_propagate_workspace.argtypes = [vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_table_set_phase_axes.argtypes = [vp, vp]
    L.redo_batched_product.argtypes = [i32, i64, vp, i32, i32, vp, i32, i32, vp, vp]
    L.redo_fidelity_grad_phase.argtypes = [vp, vp, vp, i64, i64, vp, i32, i32, i32, vp, vp, vp, vp, ctypes.c_size_t,
                                           vp, vp]
    L.redo_fidelity_grad_phase_workspace.argtypes = [vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_propagate_phase.argtypes = [vp, vp, vp, i64, i64, i32, i32, vp, vp, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_propagate_phase_workspace.argtypes = [vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_propagate_drift.argtypes = [vp, vp, vp, i64, i64, i32, i32, vp, vp, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_propagate_drift_workspace.argtypes = [vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_fidelity_grad_drift.argtypes = [vp, vp, vp, i64, i64, vp, i32, i32, i32, i32, vp, vp, vp, ctypes.c_size_t,
                                           vp, vp]
    L.redo_fidelity_grad_drift_workspace.argtypes = [vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_propagate_noalloc.argtypes = [vp, vp, i64, i64, i32, vp, vp, vp, vp, vp, vp]
    L.redo_fidelity_grad.argtypes = [vp, vp, i64, i64, vp, i32, i32, i32, i32, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_fidelity_grad_workspace.argtypes = [vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_grape_step.argtypes = [vp, vp, vp, i64, i64, dbl, vp, vp]
    L.redo_simulate.argtypes = [vp, vp, i64, i64, i32, i32, vp, i32, vp, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_simulate_workspace.argtypes = [vp, i64, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_expect_diag.argtypes = [vp, vp, i64, i64, i32, vp, vp, vp, vp, vp, vp]
    L.redo_state_grad_workspace.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_state_grad.argtypes = [vp, vp, i64, i64, i32, vp, vp, i32, vp, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_mlp_sizes.argtypes = [i32, vp, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.redo_mlp_forward.argtypes = [i32, vp, vp, vp, i64, vp, vp, vp]
    L.redo_mlp_backward.argtypes = [i32, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp]
    L.redo_mlp_adam.argtypes = [i64, vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, vp]
    L.redo_grape_adam_step.argtypes = [vp, vp, vp, vp, vp, i64, i64, i32, dbl, dbl, dbl, dbl, vp]
    L.redo_propagate_steps.argtypes = [vp, vp, i64, i64, i32, vp, vp, ctypes.c_size_t, vp, vp]
    L.redo_propagate_steps_workspace.argtypes = [vp, i64, i64, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_reunitarize.argtypes = [i32, i64, i32, vp, vp, i32, vp]
    L.redo_plan.argtypes = [dbl, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                            ctypes.POINTER(i64)]
    L.redo_grape_lbfgs_workspace.argtypes = [vp, i64, i64, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.redo_grape_lbfgs_step.argtypes = [vp, vp, vp, vp, i64, i64, i32, i32, dbl, dbl, vp, ctypes.c_size_t, vp, vp,
                                        vp]
    L.redo_profile_enable.argtypes = [i32]
    L.redo_profile_read.argtypes = [vp, vp, i32]
    L.redo_last_error.restype = ctypes.c_char_p
    L.redo_last_error.argtypes = []
    for name in EXPORTS:
        if name != "redo_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != REDO_OK:
        raise RedoError(status, load_library().redo_last_error().decode())


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


# (N, K) of every live table handle: the C ABI takes plain pointers, so the binding checks here
# that each array holds what the library will read or write for that table.
_TABLE_NK: dict = {}


def _table_nk(handle: int) -> tuple[int, int]:
    nk = _TABLE_NK.get(handle)
    if nk is None:
        info = redo_table_info(handle)
        nk = _TABLE_NK[handle] = (info["N"], info["K"])
    return nk


def _exact(t: torch.Tensor, name: str, dtype, count: int):
    """An input the library reads ``count`` elements of: that dtype and exactly that many elements."""
    if t.dtype != dtype:
        raise ValueError(f"{name}: {dtype} expected, got {t.dtype}")
    if t.numel() != count:
        raise ValueError(f"{name}: {count} elements expected for this table and shape, got {t.numel()}")


def _room(t: torch.Tensor | None, name: str, nbytes: int):
    """An array the library writes (or reads) ``nbytes`` of: at least that many bytes."""
    if t is not None and t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{name}: {nbytes} bytes needed, got {t.numel() * t.element_size()}")


def _levels(handle: int, q: torch.Tensor) -> tuple[int, int, int, int]:
    """(B, M, N, K) of a level-index array q [B][M][K] (int32) for this table, checked."""
    B, M = q.shape[0], q.shape[1]
    N, K = _table_nk(handle)
    _exact(q, "q", torch.int32, B * M * K)
    return B, M, N, K


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def redo_build_table(H0: torch.Tensor, Hk: torch.Tensor, dt: float, lo, hi, base: int, digits: int,
                     flags: int = REDO_TABLE_FP32, stream=None) -> int:
    """Build the discrete-operator table; returns the opaque handle (an int)."""
    L = load_library()
    N = H0.shape[0]
    K = Hk.shape[0]
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    if tuple(H0.shape) != (N, N) or tuple(Hk.shape) != (K, N, N):
        raise ValueError(f"H0 [N][N] and Hk [K][N][N] expected, got {tuple(H0.shape)} and {tuple(Hk.shape)}")
    if H0.dtype != torch.complex128 or Hk.dtype != torch.complex128:
        raise ValueError("H0 and Hk: torch.complex128 expected")
    if lo.size != K or hi.size != K:
        raise ValueError(f"lo and hi: {K} values expected (one per control term), got {lo.size} and {hi.size}")
    out = ctypes.c_void_p()
    _check(L.redo_build_table(N, K, float(dt), _ptr(H0), _ptr(Hk), lo.ctypes.data_as(ctypes.c_void_p),
                              hi.ctypes.data_as(ctypes.c_void_p), base, digits, flags, _stream(stream),
                              ctypes.byref(out)))
    return out.value


def redo_table_free(handle: int):
    _TABLE_NK.pop(handle, None)
    _check(load_library().redo_table_free(ctypes.c_void_p(handle)))


def redo_table_info(handle: int) -> dict:
    i = [ctypes.c_int32() for _ in range(4)]
    j = [ctypes.c_int64() for _ in range(2)]
    _check(load_library().redo_table_info(ctypes.c_void_p(handle), *[ctypes.byref(x) for x in i],
                                          *[ctypes.byref(x) for x in j]))
    return dict(N=i[0].value, K=i[1].value, base=i[2].value, digits=i[3].value, levels=j[0].value,
                entries=j[1].value)


def redo_table_copy(handle: int, table_out: torch.Tensor | None, drift_out: torch.Tensor | None, stream=None):
    i = redo_table_info(handle)
    _room(table_out, "table_out", i["entries"] * i["N"] * i["N"] * 16)
    _room(drift_out, "drift_out", i["N"] * i["N"] * 16)
    _check(load_library().redo_table_copy(ctypes.c_void_p(handle), _ptr(table_out), _ptr(drift_out),
                                          _stream(stream)))


def redo_quantize(handle: int, u: torch.Tensor, q: torch.Tensor, status: torch.Tensor | None = None, stream=None):
    B, M = u.shape[0], u.shape[1]
    N, K = _table_nk(handle)
    _exact(u, "u", torch.float64, B * M * K)
    _exact(q, "q", torch.int32, B * M * K)
    _check(load_library().redo_quantize(ctypes.c_void_p(handle), _ptr(u), B, M, _ptr(q), _ptr(status),
                                        _stream(stream)))


def redo_propagate_workspace(handle: int, B: int, M: int, prec, reunit_every: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_propagate_workspace(ctypes.c_void_p(handle), B, M, _prec(prec), reunit_every,
                                                   ctypes.byref(n)))
    return n.value


def redo_propagate(handle: int, q: torch.Tensor, prec, U_out: torch.Tensor | None, U_target: torch.Tensor | None,
                   F_out: torch.Tensor | None, tau_out: torch.Tensor | None, workspace: torch.Tensor,
                   status: torch.Tensor | None = None, reunit_every: int = 0, stream=None):
    B, M, N, K = _levels(handle, q)
    _room(U_out, "U_out", B * N * N * 16)
    _room(U_target, "U_target", N * N * 16)
    _room(F_out, "F_out", B * 8)
    _room(tau_out, "tau_out", B * 16)
    _check(load_library().redo_propagate(ctypes.c_void_p(handle), _ptr(q), B, M, _prec(prec), reunit_every,
                                         _ptr(U_out), _ptr(U_target), _ptr(F_out), _ptr(tau_out),
                                         _ptr(workspace), workspace.numel() * workspace.element_size(),
                                         _ptr(status), _stream(stream)))


def redo_batched_product(A: torch.Tensor, B: torch.Tensor, adjA: bool = False, adjB: bool = False,
                         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C_b = op(A_b) op(B_b) (complex128 on the device; a 2-D operand is used for every b)."""
    N = A.shape[-1]
    count = max(A.shape[0] if A.dim() == 3 else 1, B.shape[0] if B.dim() == 3 else 1)
    if out is None:
        out = torch.empty((count, N, N), dtype=torch.complex128, device=A.device)
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != torch.complex128 or t.dim() not in (2, 3) or tuple(t.shape[-2:]) != (N, N):
            raise ValueError(f"{name}: complex128 [N][N] or [count][N][N] with N = {N} expected, got "
                             f"{t.dtype} {tuple(t.shape)}")
    if A.dim() == 3 and B.dim() == 3 and A.shape[0] != B.shape[0]:
        raise ValueError(f"A and B batches differ: {A.shape[0]} and {B.shape[0]}")
    _room(out, "out", count * N * N * 16)
    A, B = A.contiguous(), B.contiguous()
    _check(load_library().redo_batched_product(N, count, _ptr(A), int(adjA), int(A.dim() == 3), _ptr(B), int(adjB),
                                               int(B.dim() == 3), _ptr(out), _stream(stream)))
    return out


def redo_table_set_phase_axes(handle: int, sz: np.ndarray):
    """Attach the diagonals of the species' S_kz ([K][N], host) for amplitude/phase calls."""
    sz = np.ascontiguousarray(sz, dtype=np.float64)
    N, K = _table_nk(handle)
    if sz.size != K * N:
        raise ValueError(f"sz: [K][N] = {K * N} values expected, got {sz.size}")
    _check(load_library().redo_table_set_phase_axes(ctypes.c_void_p(handle), sz.ctypes.data))


def redo_propagate_phase_workspace(handle: int, B: int, M: int, prec, reunit_every: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_propagate_phase_workspace(ctypes.c_void_p(handle), B, M, _prec(prec), reunit_every,
                                                         ctypes.byref(n)))
    return n.value


def redo_propagate_phase(handle: int, q: torch.Tensor, phi: torch.Tensor, prec, U_out: torch.Tensor | None,
                         U_target: torch.Tensor | None, F_out: torch.Tensor | None, tau_out: torch.Tensor | None,
                         workspace: torch.Tensor, status: torch.Tensor | None = None, reunit_every: int = 0,
                         stream=None):
    """Amplitude/phase controls: q the quantised amplitudes, phi [B][M][K] the phases (radians)."""
    B, M, N, K = _levels(handle, q)
    _room(phi, "phi", B * M * K * 8)
    _room(U_out, "U_out", B * N * N * 16)
    _room(F_out, "F_out", B * 8)
    _check(load_library().redo_propagate_phase(ctypes.c_void_p(handle), _ptr(q), _ptr(phi), B, M, _prec(prec),
                                               reunit_every, _ptr(U_out), _ptr(U_target), _ptr(F_out),
                                               _ptr(tau_out), _ptr(workspace),
                                               workspace.numel() * workspace.element_size(), _ptr(status),
                                               _stream(stream)))


def redo_propagate_noalloc(handle: int, q: torch.Tensor, prec, U_out: torch.Tensor | None,
                           U_target: torch.Tensor | None, F_out: torch.Tensor | None, tau_out: torch.Tensor | None,
                           status: torch.Tensor | None = None, stream=None):
    """redo_propagate without a workspace: scratch is the library's fixed device array
    (for callers that cannot allocate device memory)."""
    B, M, N, K = _levels(handle, q)
    _room(U_out, "U_out", B * N * N * 16)
    _room(F_out, "F_out", B * 8)
    _room(tau_out, "tau_out", B * 16)
    _check(load_library().redo_propagate_noalloc(ctypes.c_void_p(handle), _ptr(q), B, M, _prec(prec), _ptr(U_out),
                                                 _ptr(U_target), _ptr(F_out), _ptr(tau_out), _ptr(status),
                                                 _stream(stream)))


def redo_propagate_steps_workspace(handle: int, B: int, M: int, prec) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_propagate_steps_workspace(ctypes.c_void_p(handle), B, M, _prec(prec),
                                                         ctypes.byref(n)))
    return n.value


def redo_propagate_steps(handle: int, q: torch.Tensor, prec, U_steps: torch.Tensor,
                         workspace: torch.Tensor | None = None, status: torch.Tensor | None = None, stream=None):
    """U_steps[b][n] = the step propagator of step n of pulse b (complex128 [B][M][N][N])."""
    B, M, N, K = _levels(handle, q)
    _room(U_steps, "U_steps", B * M * N * N * 16)
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(load_library().redo_propagate_steps(ctypes.c_void_p(handle), _ptr(q), B, M, _prec(prec), _ptr(U_steps),
                                               _ptr(workspace), nbytes, _ptr(status), _stream(stream)))


def redo_reunitarize(P_in: torch.Tensor, U_out: torch.Tensor, prec="fp64", iters: int = 1, stream=None):
    """Newton-Schulz steps P <- P (3I - P^dag P)/2 on complex128 [count][N][N] matrices."""
    N = P_in.shape[-1]
    count = P_in.numel() // (N * N)
    if P_in.dtype != torch.complex128 or P_in.numel() != count * N * N:
        raise ValueError(f"P_in: complex128 [count][N][N] expected, got {P_in.dtype} {tuple(P_in.shape)}")
    _room(U_out, "U_out", count * N * N * 16)
    _check(load_library().redo_reunitarize(N, count, _prec(prec), _ptr(P_in), _ptr(U_out), int(iters),
                                           _stream(stream)))


def redo_plan(omega_max: float, eps: float, base: int) -> tuple[int, int, int, int]:
    """Section II cost model: (l, m, p, s) for a range [0, omega_max], grain eps, base b (host only)."""
    l, m, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    s = ctypes.c_int64()
    _check(load_library().redo_plan(float(omega_max), float(eps), int(base), ctypes.byref(l), ctypes.byref(m),
                                    ctypes.byref(p), ctypes.byref(s)))
    return l.value, m.value, p.value, s.value


def redo_fidelity_grad_workspace(handle: int, B: int, M: int, prec, checkpoint_every: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_fidelity_grad_workspace(ctypes.c_void_p(handle), B, M, _prec(prec), checkpoint_every,
                                                       ctypes.byref(n)))
    return n.value


def redo_fidelity_grad(handle: int, q: torch.Tensor, U_target: torch.Tensor, prec, checkpoint_every: int,
                       F_out: torch.Tensor | None, grad: torch.Tensor, workspace: torch.Tensor,
                       status: torch.Tensor | None = None, stream=None, reunit_every: int = 0):
    """F and dF/du; reunit_every > 0 (equal to checkpoint_every) re-unitarises every checkpoint segment."""
    B, M, N, K = _levels(handle, q)
    batched = 1 if U_target.dim() == 3 else 0
    _room(U_target, "U_target", (B if batched else 1) * N * N * 16)
    _room(grad, "grad", B * M * K * 8)
    _room(F_out, "F_out", B * 8)
    _check(load_library().redo_fidelity_grad(ctypes.c_void_p(handle), _ptr(q), B, M, _ptr(U_target), batched,
                                             _prec(prec), checkpoint_every, int(reunit_every), _ptr(F_out),
                                             _ptr(grad), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                             _ptr(status), _stream(stream)))


def redo_fidelity_grad_drift_workspace(handle: int, B: int, M: int, prec, checkpoint_every: int = 0) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_fidelity_grad_drift_workspace(ctypes.c_void_p(handle), B, M, _prec(prec),
                                                             checkpoint_every, ctypes.byref(n)))
    return n.value


def redo_fidelity_grad_drift(handle: int, q: torch.Tensor, h: torch.Tensor, U_target: torch.Tensor, prec,
                             checkpoint_every: int, F_out: torch.Tensor | None, grad: torch.Tensor,
                             workspace: torch.Tensor, status: torch.Tensor | None = None, stream=None,
                             reunit_every: int = 0):
    """redo_fidelity_grad with pulse b's diagonal drift h[b] (device float64 [B][N], rad/s)."""
    B, M, N, K = _levels(handle, q)
    batched = 1 if U_target.dim() == 3 else 0
    _room(h, "h", B * N * 8)
    _room(U_target, "U_target", (B if batched else 1) * N * N * 16)
    _room(grad, "grad", B * M * K * 8)
    _room(F_out, "F_out", B * 8)
    _check(load_library().redo_fidelity_grad_drift(ctypes.c_void_p(handle), _ptr(q), _ptr(h), B, M, _ptr(U_target),
                                                   batched, _prec(prec), checkpoint_every, int(reunit_every),
                                                   _ptr(F_out), _ptr(grad), _ptr(workspace),
                                                   workspace.numel() * workspace.element_size(), _ptr(status),
                                                   _stream(stream)))


def redo_grape_step(handle: int, u: torch.Tensor, grad: torch.Tensor, step: float,
                    step_scale: torch.Tensor | None = None, stream=None):
    """In place: u <- clamp(u + step * s_b * grad, lo_k, hi_k) (gradient ascent on the fidelity)."""
    B, M = u.shape[0], u.shape[1]
    N, K = _table_nk(handle)
    _exact(u, "u", torch.float64, B * M * K)
    _room(grad, "grad", B * M * K * 8)
    _room(step_scale, "step_scale", B * 8)
    _check(load_library().redo_grape_step(ctypes.c_void_p(handle), _ptr(u), _ptr(grad), B, M, float(step),
                                          _ptr(step_scale), _stream(stream)))


def redo_simulate_workspace(handle: int, B: int, M: int, prec, reunit_every: int = 0, want_U: bool = True) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_simulate_workspace(ctypes.c_void_p(handle), B, M, _prec(prec), reunit_every,
                                                  1 if want_U else 0, ctypes.byref(n)))
    return n.value


def redo_simulate(handle: int, q: torch.Tensor, prec, reunit_every: int, psi0: torch.Tensor, obs_diag: torch.Tensor,
                  expect: torch.Tensor, U_final: torch.Tensor | None, workspace: torch.Tensor | None,
                  status: torch.Tensor | None = None, stream=None):
    B, M, N, K = _levels(handle, q)
    batched = 1 if psi0.dim() == 2 else 0
    _room(psi0, "psi0", (B if batched else 1) * N * 16)
    _room(obs_diag, "obs_diag", N * 8)
    _room(expect, "expect", B * (M + 1) * 8)
    _room(U_final, "U_final", B * N * N * 16)
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().redo_simulate(ctypes.c_void_p(handle), _ptr(q), B, M, _prec(prec), reunit_every,
                                        _ptr(psi0), batched, _ptr(obs_diag), _ptr(expect), _ptr(U_final),
                                        _ptr(workspace), nbytes, _ptr(status), _stream(stream)))


def redo_expect_diag(handle: int, q: torch.Tensor, prec, rho_diag: torch.Tensor, obs_diag: torch.Tensor,
                     expect: torch.Tensor | None, expect_mean: torch.Tensor | None,
                     status: torch.Tensor | None = None, stream=None):
    B, M, N, K = _levels(handle, q)
    _check(load_library().redo_expect_diag(ctypes.c_void_p(handle), _ptr(q), B, M, _prec(prec), _ptr(rho_diag),
                                           _ptr(obs_diag), _ptr(expect), _ptr(expect_mean), _ptr(status),
                                           _stream(stream)))


def redo_state_grad_workspace(handle: int, B: int) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_state_grad_workspace(ctypes.c_void_p(handle), B, ctypes.byref(n)))
    return n.value


def redo_state_grad(handle: int, q: torch.Tensor, prec, psi0: torch.Tensor, psi_target: torch.Tensor,
                    F: torch.Tensor | None, grad: torch.Tensor | None, workspace: torch.Tensor | None,
                    status: torch.Tensor | None = None, stream=None):
    B, M, N, K = _levels(handle, q)
    batched = 1 if psi0.dim() == 2 else 0
    _room(psi0, "psi0", (B if batched else 1) * N * 16)
    _room(psi_target, "psi_target", (B if batched else 1) * N * 16)
    _room(grad, "grad", B * M * K * 8)
    _room(F, "F", B * 8)
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load_library().redo_state_grad(ctypes.c_void_p(handle), _ptr(q), B, M, _prec(prec), _ptr(psi0),
                                          _ptr(psi_target), batched, _ptr(F), _ptr(grad), _ptr(workspace), nbytes,
                                          _ptr(status), _stream(stream)))


def _sizes_arg(sizes):
    arr = (ctypes.c_int32 * len(sizes))(*[int(x) for x in sizes])
    return arr, len(sizes) - 1


def redo_mlp_sizes(sizes, batch: int) -> tuple[int, int, int]:
    arr, L = _sizes_arg(sizes)
    p, a, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().redo_mlp_sizes(L, ctypes.cast(arr, ctypes.c_void_p), batch, ctypes.byref(p),
                                         ctypes.byref(a), ctypes.byref(w)))
    return p.value, a.value, w.value


def _mlp_check(sizes, params, x, acts):
    """params, x and acts of a network of these widths for x.shape[0] samples; returns the
    (params, acts, work) float counts of redo_mlp_sizes."""
    p, a, w = redo_mlp_sizes(sizes, x.shape[0])
    _exact(params, "params", torch.float32, p)
    _exact(x, "x", torch.float32, x.shape[0] * int(sizes[0]))
    _room(acts, "acts", a * 4)
    return p, a, w


def redo_mlp_forward(sizes, params, x, acts, y, stream=None):
    arr, L = _sizes_arg(sizes)
    _mlp_check(sizes, params, x, acts)
    _room(y, "y", x.shape[0] * int(sizes[-1]) * 4)
    _check(load_library().redo_mlp_forward(L, ctypes.cast(arr, ctypes.c_void_p), _ptr(params), _ptr(x), x.shape[0],
                                           _ptr(acts), _ptr(y), _stream(stream)))


def redo_mlp_backward(sizes, params, x, acts, y_target, grads, loss, work, stream=None):
    arr, L = _sizes_arg(sizes)
    p, _, w = _mlp_check(sizes, params, x, acts)
    _exact(y_target, "y_target", torch.float32, x.shape[0] * int(sizes[-1]))
    _room(grads, "grads", p * 4)
    _room(work, "work", w * 4)
    _room(loss, "loss", 8)
    _check(load_library().redo_mlp_backward(L, ctypes.cast(arr, ctypes.c_void_p), _ptr(params), _ptr(x), x.shape[0],
                                            _ptr(acts), _ptr(y_target), _ptr(grads), _ptr(loss), _ptr(work),
                                            _stream(stream)))


def redo_mlp_adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    if params.dtype != torch.float32:
        raise ValueError(f"params: torch.float32 expected, got {params.dtype}")
    for t, name in ((grads, "grads"), (m, "m"), (v, "v")):
        _room(t, name, params.numel() * 4)
    _check(load_library().redo_mlp_adam(params.numel(), _ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(step),
                                        float(lr), float(beta1), float(beta2), float(eps), _stream(stream)))


def redo_grape_adam_step(handle: int, u, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-12,
                         stream=None):
    """In place Adam ascent on the coefficients u (clamped to each term's grid)."""
    B, M = u.shape[0], u.shape[1]
    N, K = _table_nk(handle)
    _exact(u, "u", torch.float64, B * M * K)
    for t, name in ((grad, "grad"), (m, "m"), (v, "v")):
        _room(t, name, B * M * K * 8)
    _check(load_library().redo_grape_adam_step(ctypes.c_void_p(handle), _ptr(u), _ptr(grad), _ptr(m), _ptr(v), B, M,
                                               int(step), float(lr), float(beta1), float(beta2), float(eps),
                                               _stream(stream)))


def redo_grape_lbfgs_workspace(handle: int, B: int, M: int, history: int = 8) -> int:
    n = ctypes.c_size_t()
    _check(load_library().redo_grape_lbfgs_workspace(ctypes.c_void_p(handle), B, M, history, ctypes.byref(n)))
    return n.value


def redo_grape_lbfgs_step(handle: int, u, grad, F, state, first: bool, history: int = 8, step0: float = 0.05,
                          c1: float = 1e-4, u_best=None, F_best=None, stream=None):
    """In place: u (the point just evaluated) becomes the next point of projected L-BFGS ascent."""
    B, M = u.shape[0], u.shape[1]
    N, K = _table_nk(handle)
    _exact(u, "u", torch.float64, B * M * K)
    _room(grad, "grad", B * M * K * 8)
    _room(u_best, "u_best", B * M * K * 8)
    _room(F, "F", B * 8)
    _room(F_best, "F_best", B * 8)
    _check(load_library().redo_grape_lbfgs_step(ctypes.c_void_p(handle), _ptr(u), _ptr(grad), _ptr(F), B, M,
                                                int(history), 1 if first else 0, float(step0), float(c1),
                                                _ptr(state), state.numel() * state.element_size(), _ptr(u_best),
                                                _ptr(F_best), _stream(stream)))


def redo_profile_enable(enable: bool):
    _check(load_library().redo_profile_enable(1 if enable else 0))


def redo_profile_read() -> dict:
    """Per-phase (milliseconds, launches) recorded since the last read."""
    ms = (ctypes.c_double * PROFILE_PHASES)()
    n = (ctypes.c_int64 * PROFILE_PHASES)()
    _check(load_library().redo_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p),
                                            PROFILE_PHASES))
    return {PHASE_NAMES[i]: (ms[i], n[i]) for i in range(PROFILE_PHASES) if n[i]}


def _single_target(table, target) -> torch.Tensor:
    """The one [N][N] target of a propagation call (the gradient calls take one per pulse)."""
    target = torch.as_tensor(target, dtype=torch.complex128, device=table.device).contiguous()
    if tuple(target.shape) != (table.N, table.N):
        raise ValueError(f"propagation target must be [{table.N}][{table.N}], got {tuple(target.shape)}")
    return target


class Table:
    """Owning wrapper of a redo_table built from torch tensors on the current device."""

    def __init__(self, H0, Hk, dt, lo, hi, base=64, digits=2, fp32=True, fp16x3=False, levels=False, strang=False,
                 device="cuda"):
        H0 = torch.as_tensor(H0, dtype=torch.complex128, device=device).contiguous()
        Hk = torch.as_tensor(Hk, dtype=torch.complex128, device=device).contiguous()
        flags = ((REDO_TABLE_FP32 if fp32 else 0) | (REDO_TABLE_FP16X3 if fp16x3 else 0)
                 | (REDO_TABLE_LEVELS if levels else 0) | (REDO_TABLE_STRANG if strang else 0))
        self.strang = bool(strang)
        self.handle = redo_build_table(H0, Hk, dt, lo, hi, base, digits, flags)
        self.info = redo_table_info(self.handle)
        self.N, self.K = self.info["N"], self.info["K"]
        self.device = H0.device
        self._ws = {}

    def close(self):
        if getattr(self, "handle", None):
            redo_table_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def operators(self):
        """(T, D): the FP64 table [K][digits][base][N][N] (term 0 digit 0 folded with D) and D."""
        i = self.info
        T = torch.empty((i["K"], i["digits"], i["base"], i["N"], i["N"]), dtype=torch.complex128, device=self.device)
        D = torch.empty((i["N"], i["N"]), dtype=torch.complex128, device=self.device)
        redo_table_copy(self.handle, T, D)
        return T, D

    def quantize(self, u, status=None):
        u = torch.as_tensor(u, dtype=torch.float64, device=self.device).contiguous()
        q = torch.empty(u.shape, dtype=torch.int32, device=self.device)
        redo_quantize(self.handle, u, q, status)
        return q

    def workspace(self, B, M, prec, reunit_every=0):
        nbytes = redo_propagate_workspace(self.handle, B, M, prec, reunit_every)
        key = (B, M, _prec(prec), reunit_every)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
            self._ws[key] = ws
        return ws

    def propagate(self, q, prec="fp64", target=None, want_U=True, status=None, reunit_every=0):
        B = q.shape[0]
        U = torch.empty((B, self.N, self.N), dtype=torch.complex128, device=self.device) if want_U else None
        F = tau = None
        if target is not None:
            target = _single_target(self, target)
            F = torch.empty(B, dtype=torch.float64, device=self.device)
            tau = torch.empty(B, dtype=torch.complex128, device=self.device)
        ws = self.workspace(B, q.shape[1], prec, reunit_every)
        redo_propagate(self.handle, q, prec, U, target, F, tau, ws, status, reunit_every=reunit_every)
        return U, F, tau


def _table_set_phase_axes(self, sz):
    """Diagonals [K][N] of the species' S_kz, for :meth:`propagate_phase`."""
    redo_table_set_phase_axes(self.handle, sz)


def _table_propagate_phase(self, q, phi, prec="fp64", target=None, want_U=True, status=None, reunit_every=0):
    """(U [B][N][N] or None, F or None, tau or None) for amplitude/phase controls: amplitudes
    quantised to q on this table's x-operators, phases phi [B][M][K] in radians."""
    B, M = q.shape[0], q.shape[1]
    phi = torch.as_tensor(phi, dtype=torch.float64, device=self.device).contiguous()
    U = torch.empty((B, self.N, self.N), dtype=torch.complex128, device=self.device) if want_U else None
    F = tau = None
    if target is not None:
        target = _single_target(self, target)
        F = torch.empty(B, dtype=torch.float64, device=self.device)
        tau = torch.empty(B, dtype=torch.complex128, device=self.device)
    nbytes = redo_propagate_phase_workspace(self.handle, B, M, prec, reunit_every)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
    redo_propagate_phase(self.handle, q, phi, prec, U, target, F, tau, ws, status, reunit_every=reunit_every)
    return U, F, tau


def _table_fidelity_grad_phase(self, q, phi, target, prec="fp64", checkpoint_every=0, status=None):
    """(F [B], dF/dA [B][M][K], dF/dphi [B][M][K]) for amplitude/phase controls."""
    B, M, _, _ = _levels(self.handle, q)
    phi = torch.as_tensor(phi, dtype=torch.float64, device=self.device).contiguous()
    target = torch.as_tensor(target, dtype=torch.complex128, device=self.device).contiguous()
    _room(phi, "phi", B * M * self.K * 8)
    _room(target, "target", (B if target.dim() == 3 else 1) * self.N * self.N * 16)
    F = torch.empty(B, dtype=torch.float64, device=self.device)
    gA = torch.empty((B, M, self.K), dtype=torch.float64, device=self.device)
    gP = torch.empty((B, M, self.K), dtype=torch.float64, device=self.device)
    n = ctypes.c_size_t()
    L = load_library()
    _check(L.redo_fidelity_grad_phase_workspace(ctypes.c_void_p(self.handle), B, M, _prec(prec), checkpoint_every,
                                                ctypes.byref(n)))
    ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
    _check(L.redo_fidelity_grad_phase(ctypes.c_void_p(self.handle), _ptr(q), _ptr(phi), B, M, _ptr(target),
                                      int(target.dim() == 3), _prec(prec), checkpoint_every, _ptr(F), _ptr(gA),
                                      _ptr(gP), _ptr(ws), ws.numel(), _ptr(status), _stream(None)))
    return F, gA, gP


Table.fidelity_grad_phase = _table_fidelity_grad_phase
Table.set_phase_axes = _table_set_phase_axes
Table.propagate_phase = _table_propagate_phase


def _table_propagate_drift(self, q, h, prec="fp64", target=None, want_U=True, status=None, reunit_every=0):
    """(U [B][N][N] or None, F or None, tau or None) with a diagonal drift per pulse: h [B][N] the
    drift energies (rad/s) applied each step as diag(exp(-i dt h_b)) before the table factors."""
    B, M, _, _ = _levels(self.handle, q)
    h = torch.as_tensor(h, dtype=torch.float64, device=self.device).contiguous()
    _room(h, "h", B * self.N * 8)
    U = torch.empty((B, self.N, self.N), dtype=torch.complex128, device=self.device) if want_U else None
    F = tau = None
    if target is not None:
        target = _single_target(self, target)
        F = torch.empty(B, dtype=torch.float64, device=self.device)
        tau = torch.empty(B, dtype=torch.complex128, device=self.device)
    n = ctypes.c_size_t()
    L = load_library()
    _check(L.redo_propagate_drift_workspace(ctypes.c_void_p(self.handle), B, M, _prec(prec), reunit_every,
                                            ctypes.byref(n)))
    ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
    _check(L.redo_propagate_drift(ctypes.c_void_p(self.handle), _ptr(q), _ptr(h), B, M, _prec(prec), reunit_every,
                                  _ptr(U), _ptr(target), _ptr(F), _ptr(tau), _ptr(ws), ws.numel(), _ptr(status),
                                  _stream(None)))
    return U, F, tau


def _table_fidelity_grad_drift(self, q, h, target, prec="fp64", checkpoint_every=0, status=None, reunit_every=0):
    """(F [B], dF/du [B][M][K]) with a diagonal drift per pulse (h [B][N], rad/s)."""
    B, M = q.shape[0], q.shape[1]
    h = torch.as_tensor(h, dtype=torch.float64, device=self.device).contiguous()
    target = torch.as_tensor(target, dtype=torch.complex128, device=self.device).contiguous()
    F = torch.empty(B, dtype=torch.float64, device=self.device)
    g = torch.empty((B, M, self.K), dtype=torch.float64, device=self.device)
    nbytes = redo_fidelity_grad_drift_workspace(self.handle, B, M, prec, checkpoint_every)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
    redo_fidelity_grad_drift(self.handle, q, h, target, prec, checkpoint_every, F, g, ws, status,
                             reunit_every=reunit_every)
    return F, g


Table.propagate_drift = _table_propagate_drift
Table.fidelity_grad_drift = _table_fidelity_grad_drift


def _table_fidelity_grad(self, q, target, prec="fp64", checkpoint_every=0, status=None, reunit_every=0):
    """(F [B], grad [B][M][K]) of the fidelity against `target` at levels q."""
    B, M = q.shape[0], q.shape[1]
    target = torch.as_tensor(target, dtype=torch.complex128, device=self.device).contiguous()
    F = torch.empty(B, dtype=torch.float64, device=self.device)
    g = torch.empty((B, M, self.K), dtype=torch.float64, device=self.device)
    nbytes = redo_fidelity_grad_workspace(self.handle, B, M, prec, checkpoint_every)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
    redo_fidelity_grad(self.handle, q, target, prec, checkpoint_every, F, g, ws, status, reunit_every=reunit_every)
    return F, g


Table.fidelity_grad = _table_fidelity_grad


def _table_simulate(self, q, psi0, obs_diag, prec="fp64", reunit_every=0, want_U=True, status=None):
    """(expect [B][M+1], U_final [B][N][N] or None) along the chains of levels q."""
    B, M = q.shape[0], q.shape[1]
    psi0 = torch.as_tensor(psi0, dtype=torch.complex128, device=self.device).contiguous()
    obs = torch.as_tensor(obs_diag, dtype=torch.float64, device=self.device).contiguous()
    ex = torch.empty((B, M + 1), dtype=torch.float64, device=self.device)
    U = torch.empty((B, self.N, self.N), dtype=torch.complex128, device=self.device) if want_U else None
    nbytes = redo_simulate_workspace(self.handle, B, M, prec, reunit_every, want_U)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device) if nbytes else None
    redo_simulate(self.handle, q, prec, reunit_every, psi0, obs, ex, U, ws, status)
    return ex, U


Table.simulate = _table_simulate


def _table_expect_diag(self, q, rho_diag, obs_diag, prec="fp64", series=True, status=None):
    """(expect [B][M+1] or None, mean over steps 1..M [B]) of Tr[rho(t_n) O], diagonal rho and O."""
    B, M = q.shape[0], q.shape[1]
    rho = torch.as_tensor(rho_diag, dtype=torch.float64, device=self.device).contiguous()
    obs = torch.as_tensor(obs_diag, dtype=torch.float64, device=self.device).contiguous()
    ex = torch.empty((B, M + 1), dtype=torch.float64, device=self.device) if series else None
    mean = torch.empty(B, dtype=torch.float64, device=self.device)
    redo_expect_diag(self.handle, q, prec, rho, obs, ex, mean, status)
    return ex, mean


Table.expect_diag = _table_expect_diag


def _table_state_grad(self, q, psi0, psi_target, prec="fp64", want_grad=True, status=None):
    """(F [B], grad [B][M][K] or None) of the state fidelity |<psi_T|U|psi0>|^2 at levels q;
    psi0 and psi_target of shape [N] (shared) or [B][N]."""
    B, M = q.shape[0], q.shape[1]
    p0 = torch.as_tensor(psi0, dtype=torch.complex128, device=self.device).contiguous()
    pT = torch.as_tensor(psi_target, dtype=torch.complex128, device=self.device).contiguous()
    if p0.dim() != pT.dim():
        raise ValueError("psi0 and psi_target must both be shared or both batched")
    F = torch.empty(B, dtype=torch.float64, device=self.device)
    g = torch.empty((B, M, self.K), dtype=torch.float64, device=self.device) if want_grad else None
    nbytes = redo_state_grad_workspace(self.handle, B)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device) if nbytes else None
    redo_state_grad(self.handle, q, prec, p0, pT, F, g, ws, status)
    return F, g


Table.state_grad = _table_state_grad


def new_status(device="cuda") -> torch.Tensor:
    return torch.zeros(STATUS_WORDS, dtype=torch.int64, device=device)
