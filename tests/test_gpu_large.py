"""Large-N path (N = 128 ... 1024): table, propagation, gradient and simulation
against the oracle on reduced control sets (the oracle's Pade table is the slow part)."""
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


def _reduced(idx, n, K, B, M, base=64, digits=2):
    w = inputs.config(idx, n_qubits=n, B=B, M=M, base=base, digits=digits)
    w.Hk = w.Hk[:K].copy()
    w.lo, w.hi = w.lo[:K].copy(), w.hi[:K].copy()
    w.u = w.u[:, :, :K].copy()
    return w


def _table(w):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)


def test_large_table_matches_oracle_n7():
    w = _reduced(2, 7, 2, 1, 4)                       # N=128, K=2, b=64, d=2
    t = _table(w)
    T, D = t.operators()
    To, Do = _ref.oracle_table(w)
    assert np.abs(D.cpu().numpy() - Do).max() < 1e-14
    assert np.abs(T.cpu().numpy() - _ref.folded(To, Do)).max() < 1e-13


@pytest.mark.parametrize("prec,tol,reunit", [("fp64", 1e-12, 0), ("fp32", 2e-4, 0), ("fp32", 2e-4, 8),
                                             ("fp64", 1e-12, 8)])
def test_large_propagate_matches_oracle_n7(prec, tol, reunit):
    w = _reduced(2, 7, 2, 3, 21)                      # ragged against 8-step segments
    t = _table(w)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, prec, target=w.target, reunit_every=reunit)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    assert np.abs(U.cpu().numpy() - Uo).max() < tol
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-6


def test_large_propagate_n8_other_base():
    w = _reduced(2, 8, 1, 2, 30, base=16, digits=2)   # N=256, 256 levels
    t = _table(w)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, "fp64", target=w.target)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    assert np.abs(U.cpu().numpy() - Uo).max() < 1e-12


@pytest.mark.parametrize("prec,tol,ck", [("fp64", 1e-10, 0), ("fp64", 1e-10, 4), ("fp32", 2e-4, 0)])
def test_large_gradient_matches_oracle_n7(prec, tol, ck):
    w = _reduced(2, 7, 2, 2, 9)
    t = _table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, prec, checkpoint_every=ck)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        Fo, go = O.grape_gradient(To, Do, w.Hk, w.dt, dig[b], w.target)
        assert np.abs(g.cpu().numpy()[b] - go).max() <= tol * np.abs(go).max()
        assert abs(F.cpu().numpy()[b] - Fo) < 1e-10


@pytest.mark.parametrize("n,M", [(7, 40), (9, 12)])
def test_large_simulate_matches_oracle(n, M):
    w = inputs.config(3, n_qubits=n, B=2, M=M, base=16, digits=2)   # N=128 / 512, K=1
    t = _table(w)
    q = t.quantize(w.u)
    ex, U = t.simulate(q, w.psi0, w.obs_diag, "fp64")
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        eo, Uo = O.simulate_expectation(To, Do, dig[b], w.psi0, w.obs_diag)
        assert np.abs(ex.cpu().numpy()[b] - eo).max() < 1e-12
        assert np.abs(U.cpu().numpy()[b] - Uo).max() < 1e-12


def _tc_table(w):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True)


@pytest.mark.parametrize("reunit", [0, 8])
def test_large_tc_propagate_n7(reunit):
    w = _reduced(2, 7, 2, 3, 21)
    t = _tc_table(w)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, "fp16x3", target=w.target, reunit_every=reunit)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    assert np.abs(U.cpu().numpy() - Uo).max() < 2e-4
    Fo = np.array([O.fidelity(w.target, Uo[b]) for b in range(w.B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-6


def test_large_tc_propagate_n8_and_simulate_n9():
    w = _reduced(2, 8, 1, 2, 30, base=16, digits=2)
    t = _tc_table(w)
    q = t.quantize(w.u)
    U, _, _ = t.propagate(q, "fp16x3", reunit_every=10)
    U64, _, _ = t.propagate(q, "fp64")
    assert (U - U64).abs().max().item() < 2e-4
    w = inputs.config(3, n_qubits=9, B=2, M=12, base=16, digits=2)
    t = _tc_table(w)
    q = t.quantize(w.u)
    ex, U = t.simulate(q, w.psi0, w.obs_diag, "fp16x3")
    ex64, U64 = t.simulate(q, w.psi0, w.obs_diag, "fp64")
    assert (U - U64).abs().max().item() < 2e-4
    assert (ex - ex64).abs().max().item() < 2e-5


@pytest.mark.parametrize("ck", [0, 4])
def test_large_tc_gradient_n7(ck):
    w = _reduced(2, 7, 2, 2, 9)
    t = _tc_table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, "fp16x3", checkpoint_every=ck)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        Fo, go = O.grape_gradient(To, Do, w.Hk, w.dt, dig[b], w.target)
        assert np.abs(g.cpu().numpy()[b] - go).max() <= 1e-3 * np.abs(go).max()
        assert abs(F.cpu().numpy()[b] - Fo) < 1e-6


def test_large_level_table_matches_digit_products():
    from paper_1707_02162_gb300 import redo
    w = _reduced(2, 7, 2, 2, 12, base=16, digits=2)       # N=128, 256 levels
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True, levels=True)
    assert t.info["digits"] == 1 and t.info["entries"] == w.K * w.levels
    E, _ = t.operators()
    To, Do = _ref.oracle_table(w)
    Tf = _ref.folded(To, Do)
    Eg = E.cpu().numpy()
    for qv in [0, 1, 17, 255, 130]:
        c = O.level_digits(np.array([qv]), w.base, w.digits)[0]
        for k in range(w.K):
            assert np.abs(Eg[k, 0, qv] - Tf[k, 1, c[1]] @ Tf[k, 0, c[0]]).max() < 1e-13
    q = t.quantize(w.u)
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    U64, _, _ = t.propagate(q, "fp64")
    assert np.abs(U64.cpu().numpy() - Uo).max() < 1e-12
    U16, _, _ = t.propagate(q, "fp16x3", reunit_every=6)
    assert np.abs(U16.cpu().numpy() - Uo).max() < 2e-4
    F, g = t.fidelity_grad(q, w.target, "fp16x3")
    Fo, go = O.grape_gradient(To, Do, w.Hk, w.dt, dig[0], w.target)
    assert np.abs(g.cpu().numpy()[0] - go).max() <= 1e-3 * np.abs(go).max()


def test_large_level_table_product_form_global_controls():
    """Controls with several nonzeros per row (global sums of X and Y) keep the batched
    digit-product form of the level table at N = 128."""
    from paper_1707_02162_gb300 import redo
    w = _reduced(2, 7, 2, 1, 6, base=16, digits=2)
    P = inputs.PAULI
    w.Hk = np.stack([sum(inputs.embed({i: P[c] / 2}, 7) for i in range(7)) for c in ("X", "Y")])
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, levels=True)
    E, _ = t.operators()
    To, Do = _ref.oracle_table(w)
    Tf = _ref.folded(To, Do)
    Eg = E.cpu().numpy()
    for qv in [0, 17, 255]:
        c = O.level_digits(np.array([qv]), w.base, w.digits)[0]
        for k in range(w.K):
            assert np.abs(Eg[k, 0, qv] - Tf[k, 1, c[1]] @ Tf[k, 0, c[0]]).max() < 1e-13
    q = t.quantize(w.u)
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    U64, _, _ = t.propagate(q, "fp64")
    assert np.abs(U64.cpu().numpy() - Uo).max() < 1e-12


@pytest.mark.parametrize("nb", ["256", "128"])
@pytest.mark.parametrize("ck", [0, 2])
def test_large_tc_gradient_n8(monkeypatch, nb, ck):
    """N = 256: both operand-block widths of the tensor-core sweeps, one segment per pulse
    and several (checkpoints every 2 steps), against the oracle's gradient."""
    monkeypatch.setenv("REDO_TCL_NB", nb)
    w = _reduced(2, 8, 2, 2, 5, base=16, digits=2)     # N=256, K=2, 256 levels
    t = _tc_table(w)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad(q, w.target, "fp16x3", checkpoint_every=ck)
    To, Do = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        Fo, go = O.grape_gradient(To, Do, w.Hk, w.dt, dig[b], w.target)
        assert np.abs(g.cpu().numpy()[b] - go).max() <= 1e-3 * np.abs(go).max()
        assert abs(F.cpu().numpy()[b] - Fo) < 1e-6
    U, _, _ = t.propagate(q, "fp16x3", reunit_every=2)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    assert np.abs(U.cpu().numpy() - Uo).max() < 2e-4


def test_large_tc_gradient_general_h():
    """Controls with several nonzeros per row (global X and Y on 7 qubits, N=128) take the
    sparse-row trace path of the tensor-core reverse sweep."""
    w = inputs.config(0, n_qubits=7, B=2, M=6, base=16, digits=2)
    t = _tc_table(w)
    q = t.quantize(w.u)
    for ck in (0, 3):
        F, g = t.fidelity_grad(q, w.target, "fp16x3", checkpoint_every=ck)
        To, Do = _ref.oracle_table(w)
        _, dig, _, _ = _ref.oracle_levels(w)
        for b in range(w.B):
            Fo, go = O.grape_gradient(To, Do, w.Hk, w.dt, dig[b], w.target)
            assert np.abs(g.cpu().numpy()[b] - go).max() <= 1e-3 * np.abs(go).max()
            assert abs(F.cpu().numpy()[b] - Fo) < 1e-6


def test_n1024_sampled_against_oracle():
    """Largest size (10 qubits, N=1024): two short pulses of the noisy-drive system, FP64 and the
    tensor-core path, against the oracle evaluated on just the table entries the pulses use."""
    w = inputs.config(3, n_qubits=10, B=2, M=2, base=16, digits=2)
    t = _tc_table(w)
    q = t.quantize(w.u)
    U64, _, _ = t.propagate(q, "fp64")
    U16, _, _ = t.propagate(q, "fp16x3")
    qo, dig, _, _ = _ref.oracle_levels(w)
    th = O.table_thetas(w.lo[0], w.hi[0], w.levels, w.base, w.digits)
    D = O.expm_pade13(-1j * w.dt * w.H0)
    cache = {}

    def entry(j, c):
        if (j, c) not in cache:
            cache[(j, c)] = O.expm_pade13(-1j * w.dt * th[j, c] * w.Hk[0])
        return cache[(j, c)]

    for b in range(w.B):
        U = np.eye(w.N, dtype=complex)
        for n in range(w.u.shape[1]):
            E = entry(0, dig[b, n, 0, 0])
            for j in range(1, w.digits):
                E = entry(j, dig[b, n, 0, j]) @ E
            U = E @ D @ U
        assert np.abs(U64.cpu().numpy()[b] - U).max() < 1e-12
        assert np.abs(U16.cpu().numpy()[b] - U).max() < 2e-4


def test_large_zero_steps():
    """M = 0 on the large-N paths: identity propagators, F = |Tr U_T|^2 / N^2, empty gradient."""
    w = _reduced(2, 7, 2, 2, 3)
    t = _tc_table(w)
    q = t.quantize(w.u)[:, :0].contiguous()
    for prec in ("fp64", "fp16x3"):
        U, F, _ = t.propagate(q, prec, target=w.target)
        assert (U - torch.eye(w.N, dtype=U.dtype, device=U.device)).abs().max().item() < 1e-12
        Fo = abs(np.trace(w.target)) ** 2 / w.N ** 2
        assert abs(F.cpu().numpy() - Fo).max() < 1e-12
        F2, g = t.fidelity_grad(q, w.target, prec)
        assert g.numel() == 0 and abs(F2.cpu().numpy() - Fo).max() < 1e-12
