"""GPU state simulation (Section IV) against the oracle and a closed form."""

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


def _table(w, fp16x3=False):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=fp16x3)


@pytest.mark.parametrize("n,prec,tol", [(4, "fp64", 1e-12), (4, "fp32", 2e-5), (6, "fp64", 1e-12),
                                        (3, "fp64", 1e-12), (7, "fp64", 5e-12), (7, "fp32", 2e-5)])
def test_noisy_drive_expectation_matches_oracle(n, prec, tol):
    # N = 128 (streamed states): its FP64 table comes from the large-N Taylor build, ~1e-14 per
    # operator from the oracle's Pade table, and the 240 factors of a pulse add that up linearly
    w = inputs.config(3, B=3, M=120, n_qubits=n)      # OU-noise drive, Z on qubit 0, psi0 = |0...0>
    t = _table(w)
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    q = t.quantize(w.u, st)
    ex, U = t.simulate(q, w.psi0, w.obs_diag, prec)
    torch.cuda.synchronize()
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(w.B):
        eo, Uo = O.simulate_expectation(T, D, dig[b], w.psi0, w.obs_diag)
        assert np.abs(ex.cpu().numpy()[b] - eo).max() < tol
        assert np.abs(U.cpu().numpy()[b] - Uo).max() < (1e-12 if prec == "fp64" else 2e-4)
    assert st.cpu().numpy()[2:].tolist() == [0, 0]


def test_rabi_closed_form():
    # one spin, no drift, constant drive Omega X/2 from |0>: <Z>(t) = cos(Omega_hat t)
    from paper_1707_02162_gb300 import redo
    H0 = np.zeros((2, 2), dtype=complex)
    Hk = np.array([[[0, 0.5], [0.5, 0]]], dtype=complex)
    lo, hi, dt, M = np.array([0.0]), np.array([2 * 2 * np.pi * 5e3]), 1e-6, 400
    t = redo.Table(H0, Hk, dt, lo, hi, 64, 2, fp32=True)
    u = np.full((1, M, 1), 2 * np.pi * 5e3 * 0.987)
    q = t.quantize(u)
    ex, _ = t.simulate(q, np.array([1, 0], dtype=complex), np.array([1.0, -1.0]), "fp64", want_U=False)
    qo, _, _ = O.quantize(u, lo, hi, 4096)
    om = O.level_values(qo[0, 0, 0], lo[0], hi[0], 4096)
    tt = dt * np.arange(M + 1)
    assert np.abs(ex.cpu().numpy()[0] - np.cos(om * tt)).max() < 1e-12


def test_batched_initial_states_and_norm():
    w = inputs.config(3, B=2, M=50, n_qubits=5)
    rng = np.random.default_rng(4)
    psi = rng.standard_normal((2, w.N)) + 1j * rng.standard_normal((2, w.N))
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    t = _table(w)
    q = t.quantize(w.u)
    ones = np.ones(w.N)
    ex, _ = t.simulate(q, psi, ones, "fp64", want_U=False)
    assert np.abs(ex.cpu().numpy() - 1.0).max() < 1e-12          # <I> = |psi|^2 is conserved
    ez, _ = t.simulate(q, psi, w.obs_diag, "fp64", want_U=False)
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in range(2):
        eo, _ = O.simulate_expectation(T, D, dig[b], psi[b], w.obs_diag)
        assert np.abs(ez.cpu().numpy()[b] - eo).max() < 1e-12


def test_final_propagator_with_tensor_cores_n6():
    w = inputs.config(3, B=2, M=200, n_qubits=6)
    t = _table(w, fp16x3=True)
    q = t.quantize(w.u)
    ex, U = t.simulate(q, w.psi0, w.obs_diag, "fp16x3", reunit_every=64)
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    eo, Uo = O.simulate_expectation(T, D, dig[0], w.psi0, w.obs_diag)
    assert np.abs(U.cpu().numpy()[0] - Uo).max() < 2e-4
    assert np.abs(ex.cpu().numpy()[0] - eo).max() < 2e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_streamed_simulation_many_pulses(prec, tol):
    # at least one pulse per SM takes the streamed path (a pulse per CTA, operators through
    # shared memory); fewer take the lockstep path tested above
    w = inputs.config(3, B=160, M=12, n_qubits=7)
    t = _table(w)
    q = t.quantize(w.u)
    ex, _ = t.simulate(q, w.psi0, w.obs_diag, prec, want_U=False)
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    for b in (0, 77, 159):
        eo, _ = O.simulate_expectation(T, D, dig[b], w.psi0, w.obs_diag)
        assert np.abs(ex.cpu().numpy()[b] - eo).max() < tol
