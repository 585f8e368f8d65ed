"""Symmetric (Strang) split tables: propagators, fidelity, gradient and simulation on the GPU
against the oracle's step-by-step symmetric chain (and central differences of its continuous
form for the gradient)."""
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


def _table(w, **kw):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, strang=True, **kw)


def _reduced(idx, n, K, B, M, base=16, digits=2):
    w = inputs.config(idx, n_qubits=n, B=B, M=M, base=base, digits=digits)
    w.Hk = w.Hk[:K].copy()
    w.lo, w.hi = w.lo[:K].copy(), w.hi[:K].copy()
    w.u = w.u[:, :, :K].copy()
    return w


def _oracle_strang(w):
    T, _ = _ref.oracle_table(w)
    Dh = O.half_drift(w.H0, w.dt)
    _, dig, _, _ = _ref.oracle_levels(w)
    U = np.stack([O.propagate_strang(T, Dh, dig[b]) for b in range(w.B)])
    return T, Dh, dig, U


def _continuous_fidelity(w, uhat, target):
    U = np.eye(w.N, dtype=complex)
    for row in uhat:
        U = O.strang_split_step(w.H0, w.Hk, w.dt, row) @ U
    return O.fidelity(target, U)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-4)])
def test_strang_propagate_n8(prec, tol):
    w = inputs.config(0, B=3, M=40, base=16, digits=2)
    t = _table(w)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, prec, target=w.target)
    _, _, _, Uo = _oracle_strang(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < tol
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < (1e-13 if prec == "fp64" else 1e-6)
    # the symmetric chain differs from the folded (drift-first) one
    from paper_1707_02162_gb300 import redo
    t1 = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits)
    U1, _, _ = t1.propagate(t1.quantize(w.u), "fp64")
    assert (U1 - U).abs().max().item() > 1e-4


def test_strang_propagate_tc_n64():
    w = _reduced(1, 6, 2, 2, 24)
    t = _table(w, fp16x3=True)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, "fp16x3", target=w.target, reunit_every=8)
    _, _, _, Uo = _oracle_strang(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < 2e-4
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp16x3", 2e-4)])
def test_strang_propagate_n128(prec, tol):
    w = _reduced(2, 7, 2, 2, 9)
    t = _table(w, fp16x3=True)
    q = t.quantize(w.u)
    U, _, _ = t.propagate(q, prec)
    _, _, _, Uo = _oracle_strang(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < tol


def test_strang_dense_drift_n8():
    # a drift with an x term is not diagonal: the conjugation runs as two FP64 products
    w = inputs.config(0, B=2, M=20, base=16, digits=2)
    w.H0 = w.H0 + 2 * np.pi * 800.0 * inputs.embed({1: inputs.PAULI["X"] / 2}, 3)
    t = _table(w)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, "fp64", target=w.target)
    _, _, _, Uo = _oracle_strang(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < 1e-12
    from paper_1707_02162_gb300 import redo
    with pytest.raises(redo.RedoError):
        t.simulate(q, np.eye(8)[0].astype(complex), np.ones(8), "fp64")


@pytest.mark.parametrize("prec,rel", [("fp64", 1e-6), ("fp32", 1e-3)])
def test_strang_gradient_matches_central_differences_n8(prec, rel):
    w = inputs.config(0, B=1, M=10, base=64, digits=2)
    t = _table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, prec)
    _, _, _, Uo = _oracle_strang(w)
    assert abs(F.cpu().numpy()[0] - O.fidelity(w.target, Uo[0])) < (1e-12 if prec == "fp64" else 1e-6)
    qh, _, _, _ = _ref.oracle_levels(w)
    uhat = O.level_values(qh[0], w.lo, w.hi, w.levels)
    rng = np.random.default_rng(5)
    h = 1.0                                       # rad/s; dt h = 1e-6 rad
    gg = g.cpu().numpy()[0]
    for _ in range(12):
        n, k = int(rng.integers(w.u.shape[1])), int(rng.integers(w.K))
        up, dn = uhat.copy(), uhat.copy()
        up[n, k] += h
        dn[n, k] -= h
        fd = (_continuous_fidelity(w, up, w.target) - _continuous_fidelity(w, dn, w.target)) / (2 * h)
        assert abs(gg[n, k] - fd) <= rel * np.abs(gg).max()


def test_strang_gradient_tc_n128():
    w = _reduced(2, 7, 2, 1, 6)
    t = _table(w, fp16x3=True)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, "fp16x3", checkpoint_every=2)
    F64, g64 = t.fidelity_grad(q, w.target, "fp64")
    _, _, _, Uo = _oracle_strang(w)
    assert abs(F64.cpu().numpy()[0] - O.fidelity(w.target, Uo[0])) < 1e-12
    assert abs(F.cpu().numpy()[0] - F64.cpu().numpy()[0]) < 1e-6
    qh, _, _, _ = _ref.oracle_levels(w)
    uhat = O.level_values(qh[0], w.lo, w.hi, w.levels)
    gg = g64.cpu().numpy()[0]
    for n, k in [(0, 0), (2, 1), (5, 0), (5, 1)]:
        up, dn = uhat.copy(), uhat.copy()
        up[n, k] += 1.0
        dn[n, k] -= 1.0
        fd = (_continuous_fidelity(w, up, w.target) - _continuous_fidelity(w, dn, w.target)) / 2.0
        assert abs(gg[n, k] - fd) <= 1e-6 * np.abs(gg).max()
    assert np.abs(g.cpu().numpy() - g64.cpu().numpy()).max() <= 1e-3 * np.abs(gg).max()


@pytest.mark.parametrize("n,prec,tol", [(3, "fp64", 1e-12), (7, "fp64", 1e-12), (7, "fp32", 1e-5)])
def test_strang_simulate(n, prec, tol):
    w = inputs.config(3, n_qubits=n, B=2, M=24, base=16, digits=2)
    t = _table(w)
    q = t.quantize(w.u)
    ex, U = t.simulate(q, w.psi0, w.obs_diag, prec)
    T, Dh, dig, _ = _oracle_strang(w)
    for b in range(w.B):
        eo, Uo = O.simulate_expectation_strang(T, Dh, dig[b], w.psi0, w.obs_diag)
        assert np.abs(ex.cpu().numpy()[b] - eo).max() < tol
        assert np.abs(U.cpu().numpy()[b] - Uo).max() < (1e-12 if prec == "fp64" else 2e-4)
