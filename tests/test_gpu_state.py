"""State-to-state GRAPE on the GPU (redo_state_grad) against the oracle's explicit gradient,
for the small and large-N operator layouts, batched states and symmetric-split tables."""
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


def _reduced(idx, n, K, B, M, base=16, digits=2):
    w = inputs.config(idx, n_qubits=n, B=B, M=M, base=base, digits=digits)
    w.Hk = w.Hk[:K].copy()
    w.lo, w.hi = w.lo[:K].copy(), w.hi[:K].copy()
    w.u = w.u[:, :, :K].copy()
    return w


def _states(N, B, seed):
    rng = np.random.default_rng(seed)
    p0 = rng.normal(size=(B, N)) + 1j * rng.normal(size=(B, N))
    pT = rng.normal(size=(B, N)) + 1j * rng.normal(size=(B, N))
    return p0 / np.linalg.norm(p0, axis=1, keepdims=True), pT / np.linalg.norm(pT, axis=1, keepdims=True)


def _check(w, prec, rel, batched=True, seed=3, **tkw):
    from paper_1707_02162_gb300 import redo
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, **tkw)
    q = t.quantize(w.u)
    p0, pT = _states(w.N, w.B, seed)
    if not batched:
        p0, pT = p0[0], pT[0]
    F, g = t.state_grad(q, p0, pT, prec)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        a0, aT = (p0[b], pT[b]) if batched else (p0, pT)
        Fo, go = O.state_transfer_gradient(To, Do, w.Hk, w.dt, dig[b], a0, aT)
        assert abs(F.cpu().numpy()[b] - Fo) < (1e-13 if prec == "fp64" else 1e-6)
        assert np.abs(g.cpu().numpy()[b] - go).max() <= rel * np.abs(go).max()


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-11), ("fp32", 1e-4)])
def test_state_grad_n8(prec, rel):
    _check(inputs.config(0, B=3, M=12, base=16, digits=2), prec, rel)


def test_state_grad_n8_shared_states():
    _check(inputs.config(0, B=2, M=9, base=16, digits=2), "fp64", 1e-11, batched=False)


def test_state_grad_n64():
    _check(_reduced(1, 6, 2, 2, 8), "fp64", 1e-11)


@pytest.mark.parametrize("n,prec,rel,batched", [(6, "fp32", 1e-3, False), (7, "fp32", 1e-3, True),
                                                (7, "fp64", 1e-11, True), (9, "fp32", 1e-3, True)])
def test_state_grad_streamed_sizes(n, prec, rel, batched):
    # N = 64, 128 (four row groups per chunk in the reverse pass), 512 (one column per thread)
    _check(_reduced(3, n, 1, 2, 3, base=4, digits=2), prec, rel, batched=batched)


def test_state_grad_n1024_two_columns_per_thread():
    # N = 1024: two columns per thread in the reverse pass, eight rows per 64 KB chunk, two stages
    _check(_reduced(3, 10, 1, 1, 2, base=2, digits=2), "fp32", 1e-3)


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-10), ("fp32", 1e-3)])
def test_state_grad_n256_level_table(prec, rel):
    _check(_reduced(2, 8, 2, 1, 5), prec, rel, levels=True)


def test_state_grad_symmetric_split_central_differences():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=1, M=10, base=64, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, strang=True)
    q = t.quantize(w.u)
    p0, pT = _states(w.N, 1, 7)
    F, g = t.state_grad(q, p0[0], pT[0], "fp64")
    qh, _, _, _ = _ref.oracle_levels(w)
    uhat = O.level_values(qh[0], w.lo, w.hi, w.levels)

    def fs(u):
        U = np.eye(w.N, dtype=complex)
        for row in u:
            U = O.strang_split_step(w.H0, w.Hk, w.dt, row) @ U
        return abs(np.conj(pT[0]) @ U @ p0[0]) ** 2

    assert abs(F.cpu().numpy()[0] - fs(uhat)) < 1e-12
    gg = g.cpu().numpy()[0]
    for n, k in [(0, 0), (3, 1), (9, 0), (9, 1)]:
        up, dn = uhat.copy(), uhat.copy()
        up[n, k] += 1.0
        dn[n, k] -= 1.0
        assert abs(gg[n, k] - (fs(up) - fs(dn)) / 2.0) <= 1e-6 * np.abs(gg).max()


def test_state_grad_zero_steps():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=2, M=4, base=16, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits)
    q = t.quantize(w.u)[:, :0].contiguous()
    p0, pT = _states(w.N, w.B, 11)
    F, g = t.state_grad(q, p0, pT, "fp64")
    assert g.numel() == 0
    assert np.abs(F.cpu().numpy() - np.abs(np.sum(np.conj(pT) * p0, axis=1)) ** 2).max() < 1e-14


def test_state_autograd_and_grape_loop_reach_the_state():
    from paper_1707_02162_gb300 import redo
    from paper_1707_02162_gb300.grape import RedoStateFidelity, grape
    w = inputs.config(0, B=4, M=100, base=64, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits)
    p0 = np.zeros(w.N, dtype=complex)
    p0[0] = 1.0
    # reachable targets: the states another random pulse of the same system produces
    u2 = np.random.default_rng(14).uniform(w.lo[0], w.hi[0], size=w.u.shape)
    U2, _, _ = t.propagate(t.quantize(u2), "fp64")
    pT = U2.cpu().numpy()[:, :, 0].copy()
    u = torch.tensor(w.u, dtype=torch.float64, device="cuda", requires_grad=True)
    F = RedoStateFidelity.apply(u, t, np.tile(p0, (w.B, 1)), pT, "fp64")
    F.sum().backward()
    _, g = t.state_grad(t.quantize(w.u), np.tile(p0, (w.B, 1)), pT, "fp64")
    assert torch.equal(u.grad, g)
    res = grape(t, pT, torch.tensor(w.u, device="cuda"), iters=300, step=0.02 * w.extra["Omega"],
                optimizer="adam", psi0=np.tile(p0, (w.B, 1)), threshold=0.99)
    assert (res.reached >= 0).all()
    assert res.u.max().item() <= w.hi[0] and res.u.min().item() >= w.lo[0]
