"""Re-unitarised gradient chains (redo_fidelity_grad's reunit_every) near F = 1.

Reduced-precision products lose norm coherently (~3e-8 per split-FP16 product with FP32
accumulation); over thousands of products that lowers a fidelity near 1 by far more than 1e-6.
With reunit_every = checkpoint_every every checkpoint segment is replaced by its polar factor
before tau and F are formed.  Checked against the oracle's chain and gradient on pulses whose
target sits close to their own propagator (F ~ 0.99), where the drift shows:
  * N=128 (7 qubits, 2 controls), M=2000, digit table: 8 000 split-FP16 products (tensor-core
    sweeps, kept states);
  * N=64 (6 qubits, 12 controls), M=500: 12 000 FP32 products (SIMT chains).
Bars: |F - F_oracle| <= 1e-6 with re-unitarisation (and smaller than without it).  Near the
optimum the gradient is small against its natural scale 2 dt ||H_k|| |tau| / N (the largest
|dF/du| any pulse can have at this |tau|), so its error is bounded against that scale: 1e-5 (split
FP16) or 2e-5 (FP32) of it, ~1e-3 of the largest oracle entry here.
"""
import dataclasses

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


def _near_target(rng, U, eps):
    N = U.shape[0]
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    G = (G + G.conj().T) / 2
    return U @ O.expm_hermitian(G / np.linalg.norm(G, 2), eps)


@pytest.mark.parametrize("case", ["n128_fp16x3", "n64_fp32"])
def test_reunitarised_gradient_keeps_fidelity_near_one(case):
    from paper_1707_02162_gb300 import redo
    if case == "n128_fp16x3":
        w = inputs.config(2, n_qubits=7, B=1, M=2000, base=16, digits=2)
        w.Hk, w.lo, w.hi, w.u = w.Hk[:2].copy(), w.lo[:2].copy(), w.hi[:2].copy(), w.u[:, :, :2].copy()
        prec, ck, gtol = "fp16x3", 100, 1e-5
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=False, fp16x3=True)
        T, D = _ref.LazyTable(w), O.expm_hermitian(w.H0, w.dt)
    else:
        w = inputs.config(1, B=1, M=500, base=64, digits=2)
        prec, ck, gtol = "fp32", 50, 2e-5
        t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
        T, D = _ref.oracle_table(w, method="eig")
    qo, dig, _, _ = _ref.oracle_levels(w)
    Uo = O.propagate(T, D, dig[0])
    target = _near_target(np.random.default_rng(3), Uo, 0.15)
    Fo, go = O.grape_gradient(T, D, w.Hk, w.dt, dig[0], target)
    assert 0.9 < Fo < 0.9999
    q = t.quantize(w.u)
    assert np.array_equal(q.cpu().numpy(), qo)
    F_re, g_re = t.fidelity_grad(q, target, prec, checkpoint_every=ck, reunit_every=ck)
    F_no, _ = t.fidelity_grad(q, target, prec, checkpoint_every=ck)
    d_re = abs(F_re.item() - Fo)
    d_no = abs(F_no.item() - Fo)
    assert d_re <= 1e-6
    assert d_re < d_no
    scale = 2 * w.dt * max(np.linalg.norm(h, 2) for h in w.Hk) * np.sqrt(Fo)   # |tau| / N = sqrt(F)
    assert np.abs(g_re.cpu().numpy()[0] - go).max() <= gtol * scale
    from paper_1707_02162_gb300 import redo as R
    with pytest.raises(R.RedoError):
        t.fidelity_grad(q, target, prec, checkpoint_every=ck, reunit_every=ck + 1)
    t.close()


def test_reunitarised_drift_gradient_at_the_warm_start_shape():
    """The warm-start study's call: N=32, K=10, M=500, every pulse its own diagonal drift, FP32
    chains re-unitarised every 50 steps, targets near each pulse's own propagator."""
    w = inputs.config(4, B=2, M=500)
    h = inputs.drift_diagonals(w)
    from paper_1707_02162_gb300 import redo
    t = redo.Table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    T, _ = _ref.oracle_table(dataclasses.replace(w, H0=np.zeros_like(w.H0)), method="eig")   # drift-free table
    qo, dig, _, _ = _ref.oracle_levels(w)
    rng = np.random.default_rng(9)
    targets, Fo, go = [], [], []
    for b in range(w.B):
        Db = O.expm_hermitian(np.diag(h[b]).astype(np.complex128), w.dt)
        Ub = O.propagate(T, Db, dig[b])
        targets.append(_near_target(rng, Ub, 0.15))
        F_b, g_b = O.grape_gradient(T, Db, w.Hk, w.dt, dig[b], targets[-1])
        Fo.append(F_b)
        go.append(g_b)
    targets = np.stack(targets)
    q = t.quantize(w.u)
    assert np.array_equal(q.cpu().numpy(), qo)
    F_re, g_re = t.fidelity_grad_drift(q, h, targets, "fp32", checkpoint_every=50, reunit_every=50)
    F_no, _ = t.fidelity_grad_drift(q, h, targets, "fp32", checkpoint_every=50)
    for b in range(w.B):
        assert 0.9 < Fo[b] < 0.9999
        assert abs(F_re.cpu().numpy()[b] - Fo[b]) <= 1e-6
        assert abs(F_re.cpu().numpy()[b] - Fo[b]) <= abs(F_no.cpu().numpy()[b] - Fo[b]) + 1e-9
        scale = 2 * w.dt * 0.5 * np.sqrt(Fo[b])
        assert np.abs(g_re.cpu().numpy()[b] - go[b]).max() <= 2e-5 * scale
    t.close()
