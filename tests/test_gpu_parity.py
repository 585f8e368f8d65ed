"""GPU parity: libredo (through the C ABI) against the CPU FP64 oracle.

Bars: level indices bit-exact; FP64 table <= 1e-13 and FP64 propagators
<= 1e-12 max-entry; reduced precisions within the stated bounds and
|dF| <= 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs
from tests import _ref

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-4       # max-entry, FP32 chains of up to 48 000 products
F_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _table(w, fp16x3=False):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=fp16x3)


def _status():
    from paper_1707_02162_gb300 import redo
    return redo.new_status()


# ------------------------------------------------------------------ quantizer

def test_quantize_bit_exact_edge_values():
    w = inputs.config(1, B=2, M=64)
    t = _table(w)
    L = w.levels
    delta = (w.hi - w.lo) / (L - 1)
    grid = w.lo[None, :] + np.arange(L)[:, None] * delta[None, :]
    mids = w.lo[None, :] + (np.arange(L)[:, None] + 0.5) * delta[None, :]
    rng = np.random.default_rng(0)
    special = np.array([np.nan, np.inf, -np.inf, 1e300, -1e300, 0.0, -0.0])
    parts = [grid, mids, np.nextafter(mids, np.inf), np.nextafter(mids, -np.inf),
             rng.uniform(w.lo * 1.2, w.hi * 1.2, size=(200000, w.K)),
             np.tile(special[:, None], (1, w.K))]
    u = np.concatenate(parts)[None]          # B=1, M=rows
    st = _status()
    q = t.quantize(u, st)
    torch.cuda.synchronize()
    q_ref, nn, ns = O.quantize(u, w.lo, w.hi, L)
    assert np.array_equal(q.cpu().numpy(), q_ref)
    s = st.cpu().numpy()
    assert s[0] == nn and s[1] == ns


def test_quantize_ten_million_random_bit_exact():
    w = inputs.config(0, B=1, M=8)
    t = _table(w)
    rng = np.random.default_rng(42)
    u = rng.uniform(-1.05 * w.hi[0], 1.05 * w.hi[0], size=(50, 100000, w.K))
    q = t.quantize(u).cpu().numpy()
    q_ref, _, _ = O.quantize(u, w.lo, w.hi, w.levels)
    assert np.array_equal(q, q_ref)


@pytest.mark.parametrize("base,digits", [(64, 2), (16, 5), (256, 3)])
def test_quantize_bit_exact_near_ties_offset_grids(base, digits):
    """Values at every distance from the grid's ties, on grids offset far from zero.

    The quantizer screens each value with an FP32 estimate whose error bound grows with
    |y| and with |lo| / delta; distances from 1e-10 to 0.3 of a step on both sides of every
    tie (and of every grid point) cross that bound, for offsets up to 2^17 steps.
    """
    from paper_1707_02162_gb300 import redo
    w = inputs.config(1, B=1, M=4)
    L = base ** digits
    Om = w.extra["Omega"]
    offs = np.resize(np.array([-0.5, 0.0, 3.0, 37.5, -250.0, 1e-3, 2.0 ** 17 / (L - 1), -1e4]), w.K)
    span = np.resize(np.array([2.0, 0.37, 5.0, 1.0]), w.K) * Om
    lo = offs * span
    hi = lo + span
    t = redo.Table(w.H0, w.Hk, w.dt, lo, hi, base, digits, fp32=True)
    delta = (hi - lo) / (L - 1)
    rng = np.random.default_rng(7)
    j = rng.integers(0, L - 1, size=4096)
    dist = np.concatenate([np.geomspace(1e-10, 0.3, 96), [0.0]])
    dist = np.concatenate([dist, -dist])
    parts = []
    for c in (0.5, 0.0):
        base_pts = lo[None, :] + (j[:, None] + c) * delta[None, :]
        parts.append((base_pts[:, None, :] + dist[None, :, None] * delta[None, None, :]).reshape(-1, w.K))
    parts.append(rng.uniform(lo - 0.1 * span, hi + 0.1 * span, size=(200000, w.K)))
    u = np.concatenate(parts)[None]
    st = _status()
    q = t.quantize(u, st)
    torch.cuda.synchronize()
    q_ref, nn, ns = O.quantize(u, lo, hi, L)
    assert np.array_equal(q.cpu().numpy(), q_ref)
    s = st.cpu().numpy()
    assert s[0] == nn and s[1] == ns


# ------------------------------------------------------------------ table

@pytest.mark.parametrize("idx,n", [(0, 3), (1, 6), (4, 5), (0, 1), (0, 2)])
def test_table_matches_oracle(idx, n):
    w = inputs.config(idx, B=1, M=4, n_qubits=n)
    t = _table(w)
    T, D = t.operators()
    To, Do = _ref.oracle_table(w)
    assert np.abs(D.cpu().numpy() - Do).max() < 1e-14
    assert np.abs(T.cpu().numpy() - _ref.folded(To, Do)).max() < 1e-13


def test_table_other_base_and_digits():
    w = inputs.config(0, B=1, M=4, base=16, digits=3)
    t = _table(w)
    T, D = t.operators()
    To, Do = _ref.oracle_table(w)
    assert T.shape[1:3] == (3, 16)
    assert np.abs(T.cpu().numpy() - _ref.folded(To, Do)).max() < 1e-13


def test_table_large_norm_uses_squaring():
    # dt * theta * ||H|| >> 1 exercises the scaling-and-squaring branch
    w = inputs.config(0, B=1, M=4)
    w.dt = 2e-3
    t = _table(w)
    T, D = t.operators()
    To, Do = _ref.oracle_table(w)
    assert np.abs(T.cpu().numpy() - _ref.folded(To, Do)).max() < 1e-11


def test_table_rejects_non_hermitian():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=1, M=4)
    H0 = w.H0.copy()
    H0[0, 1] = 1.0
    with pytest.raises(redo.RedoError) as e:
        redo.Table(H0, w.Hk, w.dt, w.lo, w.hi)
    assert e.value.status == 2


# ------------------------------------------------------------------ propagators

def _check_prop(w, prec, tol, pulses=None):
    t = _table(w)
    st = _status()
    q = t.quantize(w.u, st)
    U, F, tau = t.propagate(q, prec, target=w.target, status=st)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[2:].tolist() == [0, 0]
    q_ref, dig, _, _ = _ref.oracle_levels(w)
    assert np.array_equal(q.cpu().numpy(), q_ref)
    T, D = _ref.oracle_table(w)
    pulses = range(w.B) if pulses is None else pulses
    Uo = _ref.oracle_propagators(w, T, D, dig, pulses)
    Ug = U.cpu().numpy()[list(pulses)]
    err = np.abs(Ug - Uo).max()
    assert err < tol, err
    Fo = np.array([O.fidelity(w.target, Uo[i]) for i in range(len(pulses))])
    dF = np.abs(F.cpu().numpy()[list(pulses)] - Fo).max()
    assert dF < max(F_TOL, tol), dF
    return err, dF


def test_propagate_fp64_plain_redo_n3_full():
    w = inputs.config(0)                              # N=8, M=1000, B=1
    _check_prop(w, "fp64", FP64_TOL)


def test_propagate_fp64_n6_small_batch_ragged():
    w = inputs.config(1, B=3, M=37)                   # ragged: 37*24 factors
    _check_prop(w, "fp64", FP64_TOL)


@pytest.mark.parametrize("n", [1, 2, 4, 5])
def test_propagate_fp64_other_sizes(n):
    w = inputs.config(0, B=2, M=101, n_qubits=n)
    w.target = inputs.haar_unitary(np.random.default_rng(n), 2 ** n)
    _check_prop(w, "fp64", FP64_TOL)


def test_propagate_fp32_n6():
    w = inputs.config(1, B=4, M=200)
    _check_prop(w, "fp32", FP32_TOL)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_propagate_reunitarized_matches_oracle_polar(prec, tol):
    # re-unitarisation every R steps replaces each R-step block product by its
    # polar factor; for an exact (FP64) chain that is the identity map up to rounding
    w = inputs.config(1, B=3, M=50)
    t = _table(w)
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, prec, target=w.target, reunit_every=16)
    q_ref, dig, _, _ = _ref.oracle_levels(w)
    T, D = _ref.oracle_table(w)
    Uo = _ref.oracle_propagators(w, T, D, dig, range(w.B))
    assert np.abs(U.cpu().numpy() - Uo).max() < tol
    Ug = U.cpu().numpy()
    G = np.einsum("bji,bjk->bik", Ug.conj(), Ug)
    assert np.abs(G - np.eye(w.N)).max() < 1e-11


def test_propagate_zero_steps_is_identity():
    w = inputs.config(1, B=2, M=0)
    t = _table(w)
    q = torch.zeros((2, 0, w.K), dtype=torch.int32, device="cuda")
    for prec in ("fp64", "fp32"):
        U, F, _ = t.propagate(q, prec, target=w.target)
        eye = np.eye(w.N)
        assert np.abs(U.cpu().numpy() - eye).max() == 0
        assert abs(F.cpu().numpy()[0] - O.fidelity(w.target, eye)) < 1e-15


def test_bad_level_index_is_counted_not_faulted():
    w = inputs.config(0, B=1, M=10)
    t = _table(w)
    q = t.quantize(w.u).clone()
    q[0, 3, 1] = w.levels + 5
    q[0, 4, 0] = -2
    st = _status()
    U, _, _ = t.propagate(q, "fp64", status=st)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[3] >= 2
    # bad indices were replaced by level 0
    qq = q.cpu().numpy().copy()
    qq[0, 3, 1] = 0
    qq[0, 4, 0] = 0
    T, D = _ref.oracle_table(w)
    Uo = O.propagate(T, D, O.level_digits(qq, w.base, w.digits)[0])
    assert np.abs(U.cpu().numpy()[0] - Uo).max() < FP64_TOL


def test_propagate_full_size_batched_sampled_fp64_fp32():
    # the benchmark workload shape (N=64, K=12, B=256, M=2000) in the launch
    # configuration the benchmark times; the oracle checks two sampled pulses.
    w = inputs.config(1)
    t = _table(w)
    q = t.quantize(w.u)
    q_ref, dig, _, _ = _ref.oracle_levels(w)
    assert np.array_equal(q.cpu().numpy(), q_ref)
    T, D = _ref.oracle_table(w)
    pulses = [0, 255]
    Uo = _ref.oracle_propagators(w, T, D, dig, pulses)
    for prec, tol in (("fp32", FP32_TOL), ("fp64", FP64_TOL)):
        U, F, _ = t.propagate(q, prec, target=w.target)
        Ug = U.cpu().numpy()
        assert np.abs(Ug[pulses] - Uo).max() < tol
        # properties at every pulse: unitarity and F in [0, 1]
        G = np.einsum("bji,bjk->bik", Ug.conj(), Ug)
        assert np.abs(G - np.eye(w.N)).max() < (1e-11 if prec == "fp64" else 1e-3)
        Fg = F.cpu().numpy()
        assert ((Fg >= 0) & (Fg <= 1 + 1e-9)).all()
        for i, b in enumerate(pulses):
            assert abs(Fg[b] - O.fidelity(w.target, Uo[i])) < F_TOL


@pytest.mark.parametrize("controls", ["pauli", "global"])
def test_level_table_closed_form_and_product_forms(controls):
    """Single-qubit Pauli controls (one nonzero per row, H_k^2 = I/4, one of them diagonal) take
    the closed-form level operators; global sums of X take the digit-product form.  Both must
    equal the oracle's digit products."""
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=2, M=30)
    P = inputs.PAULI
    if controls == "pauli":
        w.Hk = np.stack([inputs.embed({0: P["X"] / 2}, 3), -inputs.embed({2: P["Z"] / 2}, 3)])
    else:
        w.Hk = np.stack([sum(inputs.embed({i: P["X"] / 2}, 3) for i in range(3)),
                         inputs.embed({1: P["Y"] / 2}, 3) + inputs.embed({2: P["X"] / 2}, 3)])
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, levels=True)
    E, _ = t.operators()
    To, Do = _ref.oracle_table(w)
    Tf = _ref.folded(To, Do)
    Eg = E.cpu().numpy()
    for qv in [0, 1, 63, 64, 2047, 2048, w.levels - 1]:
        c = O.level_digits(np.array([qv]), w.base, w.digits)[0]
        for k in range(w.K):
            assert np.abs(Eg[k, 0, qv] - Tf[k, 1, c[1]] @ Tf[k, 0, c[0]]).max() < 1e-13
    q = t.quantize(w.u)
    U, _, _ = t.propagate(q, "fp64")
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
    assert np.abs(U.cpu().numpy() - Uo).max() < FP64_TOL


def test_level_table_operators_are_digit_products():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=2, M=50)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, levels=True)
    E, D = t.operators()                     # [K][1][levels][N][N]
    To, Do = _ref.oracle_table(w)
    Tf = _ref.folded(To, Do)
    Eg = E.cpu().numpy()
    rng = np.random.default_rng(3)
    for qv in list(rng.integers(0, w.levels, size=30)) + [0, w.levels - 1]:
        c = O.level_digits(np.array([qv]), w.base, w.digits)[0]
        for k in range(w.K):
            assert np.abs(Eg[k, 0, qv] - Tf[k, 1, c[1]] @ Tf[k, 0, c[0]]).max() < 1e-14
    q = t.quantize(w.u)
    for prec, tol in (("fp64", FP64_TOL), ("fp32", FP32_TOL)):
        U, F, _ = t.propagate(q, prec, target=w.target)
        _, dig, _, _ = _ref.oracle_levels(w)
        Uo = _ref.oracle_propagators(w, To, Do, dig, range(w.B))
        assert np.abs(U.cpu().numpy() - Uo).max() < tol
    # the gradient works on a level table too
    Fg, g = t.fidelity_grad(q, w.target, "fp64")
    Fo, go = O.grape_gradient(To, Do, w.Hk, w.dt, O.level_digits(q.cpu().numpy(), w.base, w.digits)[0], w.target)
    assert np.abs(g.cpu().numpy()[0] - go).max() <= 1e-10 * np.abs(go).max()
