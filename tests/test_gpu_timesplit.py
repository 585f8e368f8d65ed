"""Time split on one GPU with virtual ranks: segment products, batched products and local
gradients through the C ABI, regrouped as the ranks would, against the whole pulse."""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs
from tests import _ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def test_batched_product_against_numpy():
    from paper_1707_02162_gb300 import redo
    rng = np.random.default_rng(4)
    for N in (3, 8, 64, 100):
        A = rng.standard_normal((5, N, N)) + 1j * rng.standard_normal((5, N, N))
        B = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
        Ad, Bd = torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")
        for adjA in (False, True):
            for adjB in (False, True):
                C = redo.redo_batched_product(Ad, Bd, adjA, adjB).cpu().numpy()
                a = np.conj(np.swapaxes(A, -1, -2)) if adjA else A
                b = B.conj().T if adjB else B
                assert np.abs(C - a @ b).max() < 1e-12 * N
    with pytest.raises(redo.RedoError):
        redo.redo_batched_product(Ad, Bd, out=Ad)          # output overlapping an input


@pytest.mark.parametrize("idx,n,K,B,M,G", [(0, None, None, 2, 40, 3), (1, 6, 4, 2, 17, 3), (2, 7, 2, 1, 9, 2)])
def test_virtual_ranks_match_the_whole_pulse(idx, n, K, B, M, G):
    from paper_1707_02162_gb300 import redo, timesplit
    w = inputs.config(idx, n_qubits=n, B=B, M=M, base=16, digits=2)
    if K is not None:
        w.Hk = w.Hk[:K].copy()
        w.lo, w.hi = w.lo[:K].copy(), w.hi[:K].copy()
        w.u = w.u[:, :, :K].copy()
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    ops = timesplit.LibraryOps(t, "fp64")
    q = t.quantize(w.u)
    bounds = [timesplit.segment_bounds(w.M, G, r) for r in range(G)]
    qs = [q[:, n0:n1].contiguous() for n0, n1 in bounds]
    segments = [ops.segment_product(qr) for qr in qs]
    U = timesplit.combine(ops, segments)
    Ufull, _, _ = t.propagate(q, "fp64")
    assert (U - Ufull).abs().max().item() < 1e-12
    target = torch.as_tensor(w.target, device="cuda")
    Ff, gf = t.fidelity_grad(q, target, "fp64")
    scale = gf.abs().max().item()
    for r, (n0, n1) in enumerate(bounds):
        F, g = ops.local_grad(qs[r], timesplit.local_target(ops, segments, r, target))
        assert (F - Ff).abs().max().item() < 1e-12
        assert (g - gf[:, n0:n1]).abs().max().item() <= 1e-9 * scale
    # and the oracle agrees with the whole pulse
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    assert np.abs(U.cpu().numpy()[0] - O.propagate(To, Do, dig[0])).max() < 1e-12
