"""A diagonal drift of each pulse's own (the warm-start workload: offsets nu and couplings J
drawn per instance).  The table is built with H0 = 0 and pulse b's drift enters every step as
diag(exp(-i dt h_b)); the oracle instead exponentiates each pulse's whole drift H0_b on its
own (Pade) and runs its plain chain, so the two routes share nothing but the inputs."""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _workload(n, B, M, seed=11):
    w = inputs.config(4, n_qubits=n, B=B, M=M, seed=seed, base=16, digits=2)
    return w, inputs.drift_diagonals(w)


def _table(w, **kw):
    from paper_1707_02162_gb300 import redo
    return redo.Table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, **kw)


def _oracle(w, h):
    T, _ = O.build_table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    Ds = [O.expm_pade13(-1j * w.dt * np.diag(h[b]).astype(np.complex128)) for b in range(w.B)]
    return T, Ds, dig


def _targets(w, seed=5):
    rng = np.random.default_rng(seed)
    return np.stack([inputs.haar_unitary(rng, w.Hk.shape[1]) for _ in range(w.B)])


@pytest.mark.parametrize("n,B,M,prec,tol,reunit", [(3, 3, 40, "fp64", 1e-12, 0), (3, 3, 40, "fp32", 2e-4, 0),
                                                   (3, 3, 40, "fp32", 2e-4, 8), (6, 2, 24, "fp64", 1e-12, 0),
                                                   (6, 2, 24, "fp64", 1e-12, 7), (6, 2, 24, "fp32", 2e-4, 0),
                                                   (6, 2, 150, "fp16x3", 2e-4, 64), (6, 2, 24, "fp16x3", 2e-4, 0),
                                                   (7, 2, 9, "fp64", 1e-12, 0), (7, 2, 9, "fp32", 2e-4, 3)])
def test_drift_propagate_matches_oracle(n, B, M, prec, tol, reunit):
    w, h = _workload(n, B, M)
    t = _table(w, fp32=True, fp16x3=n == 6)
    q = t.quantize(w.u)
    UT = _targets(w)[0]                      # the propagation calls take one target for all pulses
    U, F, _ = t.propagate_drift(q, h, prec, target=UT, reunit_every=reunit)
    T, Ds, dig = _oracle(w, h)
    Uo = np.stack([O.propagate(T, Ds[b], dig[b]) for b in range(B)])
    assert np.abs(U.cpu().numpy() - Uo).max() < tol
    Fo = np.array([O.fidelity(UT, Uo[b]) for b in range(B)])
    assert np.abs(F.cpu().numpy() - Fo).max() < (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("n,prec", [(3, "fp64"), (6, "fp16x3"), (7, "fp64")])
def test_shared_drift_equals_the_folded_table(n, prec):
    # the same drift on every pulse: the per-step diagonal and the drift folded into the table
    # are the same product up to rounding
    w, h = _workload(n, 2, 20)
    h[:] = h[0]
    t0 = _table(w, fp32=True, fp16x3=n == 6)
    from paper_1707_02162_gb300 import redo
    t1 = redo.Table(np.diag(h[0]).astype(np.complex128), w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True,
                    fp16x3=n == 6)
    q = t0.quantize(w.u)
    U0, _, _ = t0.propagate_drift(q, h, prec)
    U1, _, _ = t1.propagate(q, prec)
    assert (U0 - U1).abs().max().item() < (1e-12 if prec == "fp64" else 2e-4)


def test_drift_zero_steps_is_identity():
    w, h = _workload(3, 2, 0)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    U, F, _ = t.propagate_drift(q, h, "fp64", target=np.eye(8))
    assert np.abs(U.cpu().numpy() - np.eye(8)[None]).max() == 0.0
    assert np.abs(F.cpu().numpy() - 1.0).max() < 1e-15


@pytest.mark.parametrize("n,B,M,prec,ck,rel", [(3, 3, 12, "fp64", 0, 1e-10), (3, 3, 12, "fp64", 4, 1e-10),
                                               (3, 3, 12, "fp32", 0, 2e-3), (5, 2, 10, "fp64", 3, 1e-10),
                                               (6, 1, 6, "fp32", 2, 2e-3), (7, 2, 5, "fp64", 0, 1e-10),
                                               (7, 1, 5, "fp64", 2, 1e-10), (7, 1, 5, "fp32", 0, 2e-3)])
def test_drift_gradient_matches_oracle(n, B, M, prec, ck, rel):
    w, h = _workload(n, B, M)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    UT = _targets(w)
    F, g = t.fidelity_grad_drift(q, h, UT, prec, checkpoint_every=ck)
    T, Ds, dig = _oracle(w, h)
    for b in range(B):
        Fo, go = O.grape_gradient(T, Ds[b], w.Hk, w.dt, dig[b], UT[b])
        assert abs(F.cpu().numpy()[b] - Fo) < (1e-12 if prec == "fp64" else 1e-6)
        assert np.abs(g.cpu().numpy()[b] - go).max() <= rel * np.abs(go).max()


def test_drift_gradient_shared_target():
    w, h = _workload(3, 3, 10)
    t = _table(w, fp32=True)
    q = t.quantize(w.u)
    UT = _targets(w)[0]
    F, g = t.fidelity_grad_drift(q, h, UT, "fp64")
    F1, g1 = t.fidelity_grad_drift(q, h, np.broadcast_to(UT, (3, 8, 8)).copy(), "fp64")
    assert (F - F1).abs().max().item() == 0.0
    assert (g - g1).abs().max().item() == 0.0


def test_drift_errors():
    from paper_1707_02162_gb300 import redo
    w, h = _workload(3, 1, 4)
    ts = redo.Table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, strang=True)
    q = ts.quantize(w.u)
    with pytest.raises(redo.RedoError):
        ts.propagate_drift(q, h, "fp64")
    t = _table(w, fp32=True)
    w6, h6 = _workload(6, 1, 2)
    t6 = _table(w6, fp32=True, fp16x3=True)
    with pytest.raises(redo.RedoError):        # the drift gradient runs in FP64 or FP32
        t6.fidelity_grad_drift(t6.quantize(w6.u), h6, np.eye(64), "fp16x3")
    wl, hl = _workload(7, 1, 2)
    tl = _table(wl, fp32=True)
    with pytest.raises(redo.RedoError):
        tl.propagate_drift(tl.quantize(wl.u), hl, "fp16x3")
    with pytest.raises(redo.RedoError):       # no drift array with steps to take
        redo.load_library()
        redo._check(redo.load_library().redo_propagate_drift(
            redo.ctypes.c_void_p(t.handle), redo._ptr(q), None, 1, 4, 0, 0, None, None, None, None, None, 0, None,
            None))


def test_drift_grape_reaches_reachable_targets():
    # every instance its own system; targets made by other pulses on the same systems
    from paper_1707_02162_gb300 import grape
    w, h = _workload(3, 4, 30)
    t = _table(w, fp32=True)
    rng = np.random.default_rng(3)
    Om = w.extra["Omega"]
    u_t = torch.tensor(rng.uniform(-0.5 * Om, 0.5 * Om, w.u.shape), device="cuda")
    targets, _, _ = t.propagate_drift(t.quantize(u_t), h, "fp64")
    u0 = torch.tensor(rng.uniform(-0.3 * Om, 0.3 * Om, w.u.shape), device="cuda")
    res = grape.grape(t, targets, u0, iters=400, step=0.01 * Om, prec="fp64", threshold=0.99, optimizer="adam",
                      drift=h)
    assert bool((res.reached >= 0).all())
    # the drifts matter: judged on the first instance's system, the other instances' pulses miss
    # their targets (F about 0.4 for the target pulses themselves)
    q = t.quantize(res.u)
    F_own, _ = t.fidelity_grad_drift(q, h, targets, "fp64")
    F_one, _ = t.fidelity_grad_drift(q, np.broadcast_to(h[0], h.shape).copy(), targets, "fp64")
    assert F_own.min().item() > 0.95
    assert F_one[1:].max().item() < 0.9
