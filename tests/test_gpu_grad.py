"""GPU GRAPE gradient against the oracle's gradient and central finite differences.

Bars: FP64 gradient within 1e-10 of the oracle relative to max |g| (traces of
products of thousands of factors), FP32 within 2e-4; central differences of
the oracle's split model (h = 1e-6 in normalised amplitude) agree with the FP64
GPU gradient to 1e-6 relative.
"""
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


def _table(w):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)


def _oracle_grad(w, b=0):
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    return O.grape_gradient(T, D, w.Hk, w.dt, dig[b], w.target)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("ck", [0, 3])
def test_grad_matches_oracle_n3(prec, tol, ck):
    w = inputs.config(0, B=2, M=25)
    t = _table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, prec, checkpoint_every=ck)
    for b in range(w.B):
        Fo, go = _oracle_grad(w, b)
        gg = g.cpu().numpy()[b]
        assert np.abs(gg - go).max() <= tol * np.abs(go).max()
        assert abs(F.cpu().numpy()[b] - Fo) < max(1e-12, tol * 1e-2)


def test_grad_matches_oracle_n5_warm_start_shape():
    # N=32, K=10 (the learned-warm-start system), ragged checkpoints
    w = inputs.config(4, B=2, M=30)
    w.target = inputs.haar_unitary(np.random.default_rng(3), w.N)
    t = _table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, "fp64", checkpoint_every=7)
    Fo, go = _oracle_grad(w, 1)
    assert np.abs(g.cpu().numpy()[1] - go).max() <= 1e-10 * np.abs(go).max()


def test_grad_n6_batched_targets():
    w = inputs.config(1, B=2, M=6)
    rng = np.random.default_rng(12)
    targets = np.stack([inputs.haar_unitary(rng, w.N) for _ in range(w.B)])
    t = _table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, targets, "fp64")
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        Fo, go = O.grape_gradient(T, D, w.Hk, w.dt, dig[b], targets[b])
        assert np.abs(g.cpu().numpy()[b] - go).max() <= 1e-10 * np.abs(go).max()
        assert abs(F.cpu().numpy()[b] - Fo) < 1e-12


def test_grad_central_differences_20_entries():
    w = inputs.config(0, B=1, M=40)
    t = _table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, "fp64")
    g = g.cpu().numpy()[0]
    qo, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    uh = O.level_values(qo[0], w.lo, w.hi, w.levels)
    Om = w.extra["Omega"]
    h = 1e-6 * Om
    rng = np.random.default_rng(5)
    picks = [(int(rng.integers(w.M)), int(rng.integers(w.K))) for _ in range(20)]

    def Fsplit(u):
        U = np.eye(w.N, dtype=complex)
        for n in range(w.M):
            U = O.split_step(w.H0, w.Hk, w.dt, u[n]) @ U
        return O.fidelity(w.target, U)

    for n, k in picks:
        up, um = uh.copy(), uh.copy()
        up[n, k] += h
        um[n, k] -= h
        fd = (Fsplit(up) - Fsplit(um)) / (2 * h)
        assert abs(fd - g[n, k]) <= 1e-6 * np.abs(g).max() + 1e-9 / h


def test_grad_vanishes_at_reached_target():
    w = inputs.config(0, B=1, M=30)
    t = _table(w)
    q = t.quantize(w.u)
    U, _, _ = t.propagate(q, "fp64")
    target = U[0].cpu().numpy() * np.exp(0.4j)
    F, g = t.fidelity_grad(q, target, "fp64")
    assert abs(F.item() - 1) < 1e-12
    assert g.abs().max().item() < 1e-15


def test_autograd_function_and_grape_loop_improve_fidelity():
    from paper_1707_02162_gb300.grape import RedoFidelity, grape
    w = inputs.config(0, B=4, M=100)
    w.target = inputs.haar_unitary(np.random.default_rng(1), w.N)
    t = _table(w)
    u = torch.tensor(w.u, dtype=torch.float64, device="cuda", requires_grad=True)
    F = RedoFidelity.apply(u, t, w.target, "fp64", 0)
    F.sum().backward()
    q = t.quantize(w.u)
    _, g = t.fidelity_grad(q, w.target, "fp64")
    assert torch.equal(u.grad, g)
    # the chain rule through the Function with an upstream gradient that differs per pulse
    wts = torch.tensor([0.5, -2.0, 3.0, 0.0], dtype=torch.float64, device="cuda")
    u.grad = None
    F = RedoFidelity.apply(u, t, w.target, "fp64", 0)
    (F * wts).sum().backward()
    assert torch.equal(u.grad, wts[:, None, None] * g)
    res = grape(t, w.target, torch.tensor(w.u, device="cuda"), iters=60, step=2e10, prec="fp64")
    F0, F1 = res.F_history[0], res.F_history[-1]
    assert (F1 > F0).all() and F1.mean() > F0.mean() + 0.02
    # coefficients stay inside the level grid
    assert res.u.max().item() <= w.hi[0] and res.u.min().item() >= w.lo[0]
