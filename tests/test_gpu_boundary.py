"""Boundary entry points against the oracle: per-step propagators and re-unitarisation.

* ``redo_propagate_steps``: every U_n of a batch of pulses against the oracle's
  ``step_propagator`` (FP64 1e-12; FP32 2e-5 per step), the symmetric steps of a
  REDO_TABLE_STRANG table against ``strang_step_propagator`` (diagonal and dense drift), and
  the ordered product of the steps against ``redo_propagate``.
* ``redo_reunitarize`` (the Newton-Schulz step the reduced-precision chains apply) on
  perturbed unitaries P = U (I + E), E Hermitian with ||P^dag P - I|| ~ 1e-5, whose polar factor
  is U exactly, and on P = U + G with a general G, against ``O.polar_unitary``.  One step maps
  an error e of P^dag P - I to about 3e^2/4, so one FP64 step leaves ~1e-10 and three leave
  rounding; FP32 arithmetic leaves its own rounding, ~N * 6e-8.
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


def _steps(t, q, prec, B, M, N):
    from paper_1707_02162_gb300 import redo
    U = torch.empty((B, M, N, N), dtype=torch.complex128, device="cuda")
    nb = redo.redo_propagate_steps_workspace(t.handle, B, M, prec)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda") if nb else None
    st = redo.new_status()
    redo.redo_propagate_steps(t.handle, q, prec, U, ws, st)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[2:].tolist() == [0, 0]
    return U.cpu().numpy()


@pytest.mark.parametrize("idx,B,M", [(0, 3, 37), (1, 2, 9)])
def test_propagate_steps_match_oracle(idx, B, M):
    from paper_1707_02162_gb300 import redo
    w = inputs.config(idx, B=B, M=M, base=16, digits=3)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    q = t.quantize(w.u)
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    U64 = _steps(t, q, "fp64", w.B, w.M, w.N)
    U32 = _steps(t, q, "fp32", w.B, w.M, w.N)
    for b in range(w.B):
        for n in range(w.M):
            Uo = O.step_propagator(T, D, dig[b, n])
            assert np.abs(U64[b, n] - Uo).max() < 1e-12
            assert np.abs(U32[b, n] - Uo).max() < 2e-5
    # the chain is the ordered product of the steps
    Uc, _, _ = t.propagate(q, "fp64")
    for b in range(w.B):
        P = np.eye(w.N, dtype=complex)
        for n in range(w.M):
            P = U64[b, n] @ P
        assert np.abs(P - Uc.cpu().numpy()[b]).max() < 1e-12
    t.close()


@pytest.mark.parametrize("dense", [False, True])
def test_propagate_steps_symmetric_split(dense):
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=2, M=11, base=16, digits=2)
    if dense:
        w.H0 = w.H0 + 2 * np.pi * 800.0 * inputs.embed({1: inputs.PAULI["X"] / 2}, 3)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, strang=True)
    q = t.quantize(w.u)
    T, _ = _ref.oracle_table(w)
    Dh = O.half_drift(w.H0, w.dt)
    _, dig, _, _ = _ref.oracle_levels(w)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        U = _steps(t, q, prec, w.B, w.M, w.N)
        for b in range(w.B):
            for n in range(w.M):
                assert np.abs(U[b, n] - O.strang_step_propagator(T, Dh, dig[b, n])).max() < tol
    t.close()


def test_propagate_steps_rejects_large_n_and_tensor_core_precision():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(1, B=1, M=2, base=16, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True)
    q = t.quantize(w.u)
    U = torch.empty((1, 2, w.N, w.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(redo.RedoError) as e:
        redo.redo_propagate_steps(t.handle, q, "fp16x3", U)
    assert e.value.status == 5
    t.close()


def test_workspace_queries_for_an_empty_batch_at_large_n():
    # B = 0 is a valid request: the N > 64 segment plans divide the GPU among B pulses, and the
    # queries must answer (not divide by zero) for every precision and checkpoint choice
    from paper_1707_02162_gb300 import redo
    w = inputs.config(2, B=1, M=4, n_qubits=7, base=16, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True)
    assert t.N == 128
    for prec in ("fp64", "fp32", "fp16x3"):
        for reunit in (0, 2):
            assert redo.redo_propagate_workspace(t.handle, 0, 10, prec, reunit) >= 0
        for ck in (0, 2):
            assert redo.redo_fidelity_grad_workspace(t.handle, 0, 10, prec, ck) >= 0
        assert redo.redo_simulate_workspace(t.handle, 0, 10, prec, 0, want_U=True) >= 0
    with pytest.raises(redo.RedoError) as e:
        redo.redo_simulate_workspace(t.handle, -1, 10, "fp32")
    assert e.value.status == 1
    t.close()


def _perturbed(rng, N, count, eps, hermitian):
    Us = np.stack([inputs.haar_unitary(rng, N) for _ in range(count)])
    P = np.empty_like(Us)
    for i in range(count):
        G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
        if hermitian:
            E = (G + G.conj().T) / 2
            E *= eps / (2 * np.linalg.norm(E, 2))          # ||P^dag P - I|| = ||2E + E^2|| ~ eps
            P[i] = Us[i] @ (np.eye(N) + E)
        else:
            P[i] = Us[i] + (eps / (2 * np.linalg.norm(G, 2))) * G
    return Us, P


@pytest.mark.parametrize("N", [8, 64])
def test_reunitarize_matches_polar_factor(N):
    from paper_1707_02162_gb300 import redo
    rng = np.random.default_rng(N)
    count = 37
    for hermitian in (True, False):
        Us, P = _perturbed(rng, N, count, 1e-5, hermitian)
        gap = max(np.abs(p.conj().T @ p - np.eye(N)).max() for p in P)
        assert 1e-7 < gap < 1e-4
        Po = np.stack([O.polar_unitary(p) for p in P])
        if hermitian:
            assert np.abs(Po - Us).max() < 1e-13             # the polar factor of U (I + E) is U
        Pd = torch.tensor(P, device="cuda")
        for prec, iters, tol in (("fp64", 1, 1e-9), ("fp64", 3, 1e-13), ("fp32", 1, 5e-6), ("fp32", 2, 5e-6)):
            out = torch.empty_like(Pd)
            redo.redo_reunitarize(Pd, out, prec, iters)
            got = out.cpu().numpy()
            assert np.abs(got - Po).max() < tol
            if prec == "fp64" and iters == 3:
                assert max(np.abs(g.conj().T @ g - np.eye(N)).max() for g in got) < 1e-13
        # one step really improves on its input, and works in place
        out = Pd.clone()
        redo.redo_reunitarize(out, out, "fp64", 1)
        assert np.abs(out.cpu().numpy() - Po).max() < 1e-3 * np.abs(P - Po).max()
