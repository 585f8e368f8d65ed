"""redo_propagate_noalloc against redo_propagate, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc
(allocator callbacks, plug-ins that do not own device memory, real-time loops
that forbid allocation after start-up).  Its scratch is a fixed device array
inside the library, shared by every call on a device, so this test makes two
calls in a row with different inputs and checks each against the allocating
entry point.  It lives in its own file, collected last.
"""
import numpy as np
import pytest
import torch

from paper_1707_02162_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-4}


@pytest.fixture(scope="module")
def redo():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()
    from paper_1707_02162_gb300 import redo as R
    return R


def _outputs(R, B, N, dev):
    return (torch.empty((B, N, N), dtype=torch.complex128, device=dev),
            torch.empty(B, dtype=torch.float64, device=dev),
            torch.empty(B, dtype=torch.complex128, device=dev))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_workspace_path_two_calls(redo, prec):
    # B=200 FP64 pulses do not fit the scratch with the default segment count,
    # so the no-allocation plan uses fewer, longer segments than the reference call.
    w = inputs.config(1, B=200, M=80)
    dev = torch.device("cuda")
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    target = torch.as_tensor(w.target, device=dev)
    rng = np.random.default_rng(77)
    for call in range(2):
        u = w.u if call == 0 else rng.uniform(w.lo[0], w.hi[0], size=w.u.shape)
        q = t.quantize(u)
        st_a, st_b = redo.new_status(dev), redo.new_status(dev)
        Ua, Fa, ta = _outputs(redo, w.B, w.N, dev)
        Ub, Fb, tb = _outputs(redo, w.B, w.N, dev)
        redo.redo_propagate(t.handle, q, prec, Ua, target, Fa, ta, t.workspace(w.B, w.M, prec), st_a)
        redo.redo_propagate_noalloc(t.handle, q, prec, Ub, target, Fb, tb, st_b)
        torch.cuda.synchronize()
        assert st_b.cpu().tolist() == st_a.cpu().tolist()
        assert (Ua - Ub).abs().max().item() < TOL[prec]
        assert (Fa - Fb).abs().max().item() < 1e-6
        assert (ta - tb).abs().max().item() < w.N * TOL[prec]
    t.close()


@pytest.mark.parametrize("dense_drift", [False, True])
def test_noalloc_symmetric_split_matches_workspace_path(redo, dense_drift):
    # A symmetric-split table conjugates the pulse products by the half drift; with a drift
    # that is not diagonal that takes a second FP64 buffer inside the scratch array.
    w = inputs.config(0, B=3, M=40, base=16, digits=2)
    if dense_drift:
        w.H0 = w.H0 + 2 * np.pi * 800.0 * inputs.embed({1: inputs.PAULI["X"] / 2}, 3)
    dev = torch.device("cuda")
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, strang=True)
    plain = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    target = torch.as_tensor(w.target, device=dev)
    q = t.quantize(w.u)
    for prec in ("fp64", "fp32"):
        for _ in range(2):
            Ua, Fa, ta = _outputs(redo, w.B, w.N, dev)
            Ub, Fb, tb = _outputs(redo, w.B, w.N, dev)
            redo.redo_propagate(t.handle, q, prec, Ua, target, Fa, ta, t.workspace(w.B, w.M, prec))
            redo.redo_propagate_noalloc(t.handle, q, prec, Ub, target, Fb, tb)
            torch.cuda.synchronize()
            assert (Ua - Ub).abs().max().item() < TOL[prec]
            assert (Fa - Fb).abs().max().item() < 1e-6
        # and it is the symmetric chain, not the drift-first one
        Uc, _, _ = plain.propagate(q, prec)
        assert (Uc - Ub).abs().max().item() > 1e-4
    t.close()
    plain.close()


def test_noalloc_rejects_requests_beyond_its_scratch(redo):
    w = inputs.config(1, B=1, M=4)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    B = 4096                                    # 4096 FP64 64x64 products alone need 256 MiB
    q = torch.zeros((B, 4, w.K), dtype=torch.int32, device="cuda")
    U = torch.empty((B, w.N, w.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(redo.RedoError) as e:
        redo.redo_propagate_noalloc(t.handle, q, "fp64", U, None, None, None)
    assert e.value.status == 1 and "REDO_NOALLOC_SCRATCH_BYTES" in str(e.value)
    t.close()
