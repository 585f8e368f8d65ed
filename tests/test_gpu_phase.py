"""Amplitude/phase controls (Section III, Eq. vn): one x-table per species, the phases as the
diagonal rotation Z_n around each step's control factors.  GPU propagators through the C ABI
against the oracle's step-by-step chain U_n = Z_n E_n Z_n^dag D."""
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
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, **kw)
    t.set_phase_axes(w.extra["sz"])
    return t


def _oracle(w, pulses=None):
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    pulses = range(w.B) if pulses is None else pulses
    U = np.stack([O.propagate_phase(T, D, dig[b], w.extra["phi"][b], w.extra["sz"]) for b in pulses])
    return U


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-4)])
def test_phase_propagate_n8(prec, tol):
    w = inputs.phase_config(3, B=3, M=40, base=16, digits=2)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    U, F, _ = t.propagate_phase(q, w.extra["phi"], prec, target=w.target)
    Uo = _oracle(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < tol
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec,tol,reunit", [("fp64", 1e-12, 0), ("fp64", 1e-12, 7), ("fp32", 2e-4, 0),
                                             ("fp16x3", 2e-4, 8), ("fp16x3", 2e-4, 0)])
def test_phase_propagate_n64(prec, tol, reunit):
    w = inputs.phase_config(6, B=2, M=24, base=16, digits=2)
    t = _table(w, fp32=True, fp16x3=True)
    q = t.quantize(w.u)
    U, F, _ = t.propagate_phase(q, w.extra["phi"], prec, target=w.target, reunit_every=reunit)
    Uo = _oracle(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < tol
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < (1e-13 if prec == "fp64" else 1e-6)


def test_phase_propagate_n64_level_table_tc():
    # level table (one factor per species and step) and a pulse long enough for several segments
    w = inputs.phase_config(6, B=3, M=150, base=16, digits=2)
    t = _table(w, fp32=True, fp16x3=True, levels=True)
    q = t.quantize(w.u)
    U, F, _ = t.propagate_phase(q, w.extra["phi"], "fp16x3", target=w.target, reunit_every=64)
    Uo = _oracle(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < 2e-4
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-6


@pytest.mark.parametrize("prec,tol,reunit", [("fp64", 1e-12, 0), ("fp32", 2e-4, 0), ("fp32", 2e-4, 3)])
def test_phase_propagate_n128(prec, tol, reunit):
    w = inputs.phase_config(7, B=2, M=9, base=16, digits=2)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    U, _, _ = t.propagate_phase(q, w.extra["phi"], prec, reunit_every=reunit)
    Uo = _oracle(w)
    assert np.abs(U.cpu().numpy() - Uo).max() < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp16x3", 2e-4)])
def test_phase_zero_equals_x_only_chain(prec, tol):
    w = inputs.phase_config(6, B=2, M=20, base=16, digits=2)
    t = _table(w, fp32=True, fp16x3=True)
    q = t.quantize(w.u)
    U0, _, _ = t.propagate_phase(q, np.zeros_like(w.extra["phi"]), prec)
    U1, _, _ = t.propagate(q, prec)
    assert (U0 - U1).abs().max().item() < tol


def test_phase_zero_steps_is_identity():
    w = inputs.phase_config(3, B=2, M=0, base=16, digits=2)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    U, F, _ = t.propagate_phase(q, w.extra["phi"], "fp64", target=np.eye(8))
    assert np.abs(U.cpu().numpy() - np.eye(8)[None]).max() == 0.0
    assert np.abs(F.cpu().numpy() - 1.0).max() < 1e-15


def test_phase_errors():
    from paper_1707_02162_gb300 import redo
    w = inputs.phase_config(3, B=1, M=4, base=16, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    q = t.quantize(w.u)
    with pytest.raises(redo.RedoError):                      # no phase axes yet
        t.propagate_phase(q, w.extra["phi"], "fp64")
    # a drift with an x term does not commute with S_z of qubit 1
    H0 = w.H0 + 2 * np.pi * 300.0 * inputs.embed({1: inputs.PAULI["X"] / 2}, 3)
    t2 = redo.Table(H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits)
    with pytest.raises(redo.RedoError):
        t2.set_phase_axes(w.extra["sz"])
    # ... but it commutes with S_z of the other qubits
    t2.set_phase_axes(w.extra["sz"] * np.array([1.0, 0.0, 1.0])[:, None])
    ts = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, strang=True)
    ts.set_phase_axes(w.extra["sz"])
    with pytest.raises(redo.RedoError):
        ts.propagate_phase(q, w.extra["phi"], "fp64")


@pytest.mark.parametrize("n,B,M,prec,ck,rel", [(3, 2, 12, "fp64", 0, 1e-10), (3, 2, 12, "fp64", 4, 1e-10),
                                               (3, 2, 12, "fp32", 0, 2e-3), (6, 1, 6, "fp64", 2, 1e-10),
                                               (7, 2, 5, "fp64", 0, 1e-10), (7, 1, 5, "fp64", 2, 1e-10),
                                               (7, 1, 5, "fp32", 0, 2e-3)])
def test_phase_gradient_matches_oracle(n, B, M, prec, ck, rel):
    w = inputs.phase_config(n, B=B, M=M, base=16, digits=2)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    F, gA, gP = t.fidelity_grad_phase(q, w.extra["phi"], w.target, prec, checkpoint_every=ck)
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(B):
        Fo, gAo, gPo = O.phase_gradient(T, D, w.Hk, w.extra["sz"], w.dt, dig[b], w.extra["phi"][b], w.target)
        assert abs(F.cpu().numpy()[b] - Fo) < (1e-12 if prec == "fp64" else 1e-6)
        assert np.abs(gA.cpu().numpy()[b] - gAo).max() <= rel * np.abs(gAo).max()
        assert np.abs(gP.cpu().numpy()[b] - gPo).max() <= rel * np.abs(gPo).max()


def test_phase_gradient_zero_phase_is_the_x_gradient():
    w = inputs.phase_config(4, B=2, M=15, base=16, digits=2)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    F, gA, _ = t.fidelity_grad_phase(q, np.zeros_like(w.extra["phi"]), w.target, "fp64")
    F1, g1 = t.fidelity_grad(q, w.target, "fp64")
    assert (F - F1).abs().max().item() < 1e-13
    assert (gA - g1).abs().max().item() <= 1e-12 * g1.abs().max().item()


def test_phase_gradient_refuses_split_fp16():
    from paper_1707_02162_gb300 import redo
    w = inputs.phase_config(7, B=1, M=2, base=16, digits=2)
    t = _table(w, fp32=True, fp16x3=True)
    q = t.quantize(w.u)
    with pytest.raises(redo.RedoError):
        t.fidelity_grad_phase(q, w.extra["phi"], w.target, "fp16x3")


def test_phase_grape_reaches_a_reachable_target():
    # targets made by other amplitude/phase pulses of the same system; Adam on (A, phi) through
    # the autograd function
    from paper_1707_02162_gb300 import grape
    w = inputs.phase_config(3, B=2, M=30, base=64, digits=2)
    t = _table(w, fp32=True)
    rng = np.random.default_rng(9)
    a_t = torch.tensor(rng.uniform(0, w.hi[0], w.u.shape), device="cuda")
    p_t = torch.tensor(rng.uniform(0, 2 * np.pi, w.u.shape), device="cuda")
    targets, _, _ = t.propagate_phase(t.quantize(a_t), p_t, "fp64")
    amp = torch.tensor(w.u, device="cuda", requires_grad=True)
    phi = torch.tensor(w.extra["phi"], device="cuda", requires_grad=True)
    opt = torch.optim.Adam([{"params": [amp], "lr": 0.02 * w.hi[0]}, {"params": [phi], "lr": 0.05}])
    F0 = None
    for it in range(300):
        F = grape.RedoPhaseFidelity.apply(amp, phi, t, targets, "fp64")
        if F0 is None:
            F0 = F.detach().clone()
        opt.zero_grad()
        (-F.sum()).backward()
        opt.step()
        with torch.no_grad():
            amp.clamp_(float(w.lo[0]), float(w.hi[0]))
        if F.min().item() > 0.99:
            break
    assert F.min().item() > 0.99 > F0.max().item()
