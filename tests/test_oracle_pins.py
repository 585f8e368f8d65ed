"""Pins for the CPU oracle: closed forms, printed values, invariants, brute force.

Each test ties an oracle function to something other than itself, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")
SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)


def _rand_herm(rng, N, scale=1.0):
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    return scale * (A + A.conj().T) / 2


# ---------------------------------------------------------------- quantizer

def test_quantize_grid_points_exact():
    L = 4096
    lo, hi = np.array([-2 * np.pi * 1e4]), np.array([2 * np.pi * 1e4])
    delta = (hi[0] - lo[0]) / (L - 1)
    q = np.arange(L)
    u = (lo[0] + q * delta)[:, None]
    qq, nn, ns = O.quantize(u, lo, hi, L)
    assert nn == 0 and ns == 0
    assert np.array_equal(qq[:, 0], q)


def test_quantize_ties_half_even_and_clamp():
    # lo=0, delta=1 makes (u-lo)/delta exact, so u=q+0.5 is an exact tie.
    L = 16
    lo, hi = np.array([0.0]), np.array([15.0])
    u = np.array([0.5, 1.5, 2.5, 3.5, 14.5, -0.4, -0.6, 15.4, 15.6, -1e300, 1e300,
                  np.nan, np.inf, -np.inf])[:, None]
    q, nn, ns = O.quantize(u, lo, hi, L)
    assert list(q[:, 0]) == [0, 2, 2, 4, 14, 0, 0, 15, 15, 0, 15, 0, 0, 0]
    assert nn == 3
    # -0.6 -> -1, 15.6 -> 16, -1e300, 1e300 saturate; -0.4 -> -0 and 15.4 -> 15 do not
    assert ns == 4


def test_quantize_matches_python_scalar_brute_force():
    # Independent scalar restatement with Python floats (IEEE double) and
    # Python's round() (ties to even).
    rng = np.random.default_rng(11)
    L = 4096
    lo = np.array([-3.7, 0.0, -1e4])
    hi = np.array([5.1, 2.0, 2e4])
    u = rng.uniform(lo - 0.1 * (hi - lo), hi + 0.1 * (hi - lo), size=(2000, 3))
    # also points within +-1 ulp of midpoints
    delta = (hi - lo) / (L - 1)
    mids = lo + (np.arange(100)[:, None] + 0.5) * delta
    u = np.concatenate([u, mids, np.nextafter(mids, np.inf), np.nextafter(mids, -np.inf)])
    q, _, _ = O.quantize(u, lo, hi, L)
    for i in range(u.shape[0]):
        for k in range(3):
            d = (float(hi[k]) - float(lo[k])) / float(L - 1)
            x = (float(u[i, k]) - float(lo[k])) / d
            r = min(max(round(x), 0), L - 1)
            assert q[i, k] == r


def test_digits_worked_example():
    g = json.load(open(GOLDEN))["coarse_grain_example"]
    d = O.level_digits(np.array([g["max_level"]]), g["base"], 3)
    assert list(d[0]) == g["max_level_digits"]
    rng = np.random.default_rng(0)
    q = rng.integers(0, 64 ** 3, size=1000)
    dd = O.level_digits(q, 64, 3)
    assert np.array_equal(dd[:, 0] + 64 * dd[:, 1] + 4096 * dd[:, 2], q)
    assert dd.min() >= 0 and dd.max() <= 63


@pytest.mark.parametrize("key", ["coarse_grain_example", "freezing_grain"])
def test_cost_model_printed_values(key):
    g = json.load(open(GOLDEN))[key]
    l, m, p, s = O.plan_digits(g["omega_max"], g["eps"], g["base"])
    assert (l, m, p, s) == (g["l"], g["m"], g["p"], g["s"])


def test_table_thetas_sum_to_level_value():
    lo, hi, L, b, d = -7.0, 11.0, 4096, 64, 2
    th = O.table_thetas(lo, hi, L, b, d)
    q = np.arange(L)
    dig = O.level_digits(q, b, d)
    s = th[0, dig[:, 0]] + th[1, dig[:, 1]]
    assert np.allclose(s, O.level_values(q, np.array(lo), np.array(hi), L), rtol=0, atol=1e-13)


# ---------------------------------------------------------------- expm

@pytest.mark.parametrize("theta", [0.0, 1e-3, 0.3, 1.7, 12.0, 250.0])
def test_expm_pauli_closed_form(theta):
    ref = math.cos(theta) * I2 - 1j * math.sin(theta) * SX
    assert np.abs(O.expm_pade13(-1j * theta * SX) - ref).max() < 1e-13 * max(1, theta)
    assert np.abs(O.expm_hermitian(SX, theta) - ref).max() < 1e-13 * max(1, theta)
    refy = math.cos(theta) * I2 - 1j * math.sin(theta) * SY
    assert np.abs(O.expm_pade13(-1j * theta * SY) - refy).max() < 1e-13 * max(1, theta)


def test_expm_collective_x_is_tensor_power():
    n, th = 3, 0.77
    Hx = inputs.controls_global_xy(n)[0]
    one = math.cos(th / 2) * I2 - 1j * math.sin(th / 2) * SX
    ref = np.kron(np.kron(one, one), one)
    assert np.abs(O.expm_pade13(-1j * th * Hx) - ref).max() < 1e-14


def test_expm_diagonal_drift_exact():
    w = inputs.config(0)
    dt = w.dt
    ref = np.diag(np.exp(-1j * dt * np.real(np.diag(w.H0))))
    assert np.abs(O.expm_pade13(-1j * dt * w.H0) - ref).max() < 1e-15
    assert np.abs(O.expm_hermitian(w.H0, dt) - ref).max() < 1e-15


def test_expm_against_scipy_and_eig():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(5)
    for N, scale in [(4, 0.1), (8, 1.0), (16, 3.0), (32, 20.0)]:
        H = _rand_herm(rng, N, scale)
        A = -1j * H
        E1 = O.expm_pade13(A)
        E2 = O.expm_hermitian(H, 1.0)
        E3 = scipy_linalg.expm(A)
        tol = 1e-13 * max(1.0, scale * N)
        assert np.abs(E1 - E3).max() < tol
        assert np.abs(E1 - E2).max() < tol
        assert np.abs(E1.conj().T @ E1 - np.eye(N)).max() < tol


def test_expm_group_property():
    rng = np.random.default_rng(6)
    H = _rand_herm(rng, 8)
    a, b = 0.37, -1.21
    lhs = O.expm_pade13(-1j * a * H) @ O.expm_pade13(-1j * b * H)
    assert np.abs(lhs - O.expm_pade13(-1j * (a + b) * H)).max() < 1e-13


def test_expm_nonhermitian_general():
    # Pade path is for general matrices: nilpotent Jordan block has exp = I + A + A^2/2
    A = np.array([[0, 2.0, 0], [0, 0, 3.0], [0, 0, 0]], dtype=complex)
    ref = np.eye(3) + A + A @ A / 2
    assert np.abs(O.expm_pade13(A) - ref).max() < 1e-14


# ---------------------------------------------------------------- table & product

def _small_workload(idx=0, M=12, B=1, n=None, L_base=64, digits=2):
    return inputs.config(idx, M=M, B=B, n_qubits=n, base=L_base, digits=digits)


def test_table_group_property_and_methods_agree():
    w = _small_workload(0)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    T2, D2 = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits, method="eig")
    assert np.abs(T - T2).max() < 1e-13 and np.abs(D - D2).max() < 1e-14
    rng = np.random.default_rng(1)
    for q in rng.integers(0, w.levels, size=20):
        c = O.level_digits(np.array([q]), w.base, w.digits)[0]
        for k in range(w.K):
            prod = T[k, 1, c[1]] @ T[k, 0, c[0]]
            uh = O.level_values(q, w.lo[k], w.hi[k], w.levels)
            assert np.abs(prod - O.expm_hermitian(w.Hk[k], w.dt * uh)).max() < 1e-13


def test_commuting_case_has_no_splitting_error():
    # Z-only controls commute with a diagonal drift: the REDO product equals the
    # unsplit exponential of the quantised Hamiltonian.
    n = 2
    rng = np.random.default_rng(2)
    H0 = inputs.drift_zz(n, rng.uniform(-5e3, 5e3, n), np.array([[0, 150.0], [0, 0]]))
    Hk = np.stack([inputs.embed({0: SZ / 2}, n), inputs.embed({1: SZ / 2}, n)])
    lo, hi, L, b, d, dt = np.array([-6e4, -6e4]), np.array([6e4, 6e4]), 4096, 64, 2, 1e-6
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, b, d)
    u = rng.uniform(-6e4, 6e4, size=(1, 30, 2))
    q, _, _ = O.quantize(u, lo, hi, L)
    dig = O.level_digits(q, b, d)
    U = O.propagate(T, D, dig[0])
    uh = O.level_values(q[0], lo, hi, L)
    Htot = 30 * H0 + np.tensordot(uh.sum(axis=0), Hk, axes=1)
    assert np.abs(U - O.expm_hermitian(Htot, dt)).max() < 1e-12


def test_per_instance_diagonal_drift_enters_through_the_drift_factor_only():
    # Each warm-start instance has its own diagonal drift h_b (offsets and couplings).  The
    # operator table does not depend on H0, the drift factor is the closed form
    # diag(exp(-i dt h_b)), and the chain with that factor is the split model at the level
    # values: so one table built with H0 = 0 serves every instance.
    w = inputs.config(4, n_qubits=3, B=2, M=12, seed=11, base=16, digits=2)
    h = inputs.drift_diagonals(w)
    T0, D0 = O.build_table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    assert np.abs(D0 - np.eye(8)).max() < 1e-15
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    for b in range(2):
        H0b = np.diag(h[b]).astype(complex)
        assert np.abs(H0b - inputs.drift_zz(3, w.extra["nu"][b], w.extra["J"][b])).max() == 0.0
        Tb, Db = O.build_table(H0b, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
        assert np.array_equal(Tb, T0)
        assert np.abs(Db - np.diag(np.exp(-1j * w.dt * h[b]))).max() < 1e-14
        uh = O.level_values(q[b], w.lo, w.hi, w.levels)
        ref = np.eye(8, dtype=complex)
        for n in range(w.M):
            ref = O.split_step(H0b, w.Hk, w.dt, uh[n]) @ ref
        assert np.abs(O.propagate(T0, Db, dig[b]) - ref).max() < 1e-12
    assert np.abs(h[0] - h[1]).max() > 1e3         # the instances really differ


def test_dirac_frame_step_equals_split_step():
    # Section III: U_n = V(dt) exp(-i Omega dt S~), S~ = V^dag(dt) S V(dt)
    rng = np.random.default_rng(3)
    n = 2
    H0 = inputs.drift_zz(n, rng.uniform(-5e3, 5e3, n), np.array([[0, 180.0], [0, 0]]))
    S = inputs.controls_global_xy(n)[0]
    dt, Om = 5e-6, 4.3e4
    V = O.expm_hermitian(H0, dt)
    Stil = V.conj().T @ S @ V
    paper = V @ O.expm_pade13(-1j * Om * dt * Stil)
    ours = O.split_step(H0, S[None], dt, np.array([Om]))
    assert np.abs(paper - ours).max() < 1e-13


def test_splitting_error_is_first_order():
    rng = np.random.default_rng(4)
    n = 1
    H0 = 2 * np.pi * 3e3 * SZ / 2
    Hk = np.stack([SX / 2, SY / 2])
    errs = []
    for dt in [4e-6, 2e-6, 1e-6]:
        u = np.array([5e4, -3e4])
        errs.append(np.abs(O.split_step(H0, Hk, dt, u) - O.exact_step(H0, Hk, dt, u)).max())
    # local error of Lie-Trotter is O(dt^2): halving dt quarters it
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_strang_local_error_is_third_order():
    # symmetric placement of the drift around one control (or commuting controls): the
    # one-step error drops by 8 when dt halves.  Non-commuting controls keep their own
    # first-order ordering error; the symmetric step removes the drift's part only.
    n = 1
    H0 = 2 * np.pi * 3e3 * SZ / 2
    Hk = np.stack([SX / 2])
    u = np.array([5e4])
    errs = [np.abs(O.strang_split_step(H0, Hk, dt, u) - O.exact_step(H0, Hk, dt, u)).max()
            for dt in [4e-6, 2e-6, 1e-6]]
    assert 7.0 < errs[0] / errs[1] < 9.0 and 7.0 < errs[1] / errs[2] < 9.0


def test_strang_global_error_is_second_order():
    # fixed total time, constant controls: exact = exp(-i t_f (H0 + u.H)); the symmetric
    # chain's error quarters when the number of steps doubles (the Lie chain's halves)
    H0 = 2 * np.pi * 3e3 * SZ / 2
    Hk = np.stack([SX / 2])
    u, tf = np.array([4e4]), 40e-6
    exact = O.expm_pade13(-1j * tf * (H0 + np.tensordot(u, Hk, axes=1)))
    es, el = [], []
    for M in (10, 20, 40):
        dt = tf / M
        S = np.linalg.matrix_power(O.strang_split_step(H0, Hk, dt, u), M)
        L = np.linalg.matrix_power(O.split_step(H0, Hk, dt, u), M)
        es.append(np.abs(S - exact).max())
        el.append(np.abs(L - exact).max())
    assert 3.6 < es[0] / es[1] < 4.4 and 3.6 < es[1] / es[2] < 4.4
    assert 1.7 < el[0] / el[1] < 2.3


def test_strang_step_is_time_reversible():
    # S(dt) S(-dt) = I for one control (a drift placed on one side only fails this)
    rng = np.random.default_rng(11)
    n = 2
    H0 = inputs.drift_zz(n, rng.uniform(-5e3, 5e3, n), np.array([[0, 150.0], [0, 0]]))
    Hk = inputs.controls_global_xy(n)[:1]
    u, dt = np.array([3.1e4]), 3e-6
    P = O.strang_split_step(H0, Hk, dt, u) @ O.strang_split_step(H0, Hk, -dt, u)
    assert np.abs(P - np.eye(4)).max() < 1e-13
    L = O.split_step(H0, Hk, dt, u) @ O.split_step(H0, Hk, -dt, u)
    assert np.abs(L - np.eye(4)).max() > 1e-4


def test_strang_table_chain_matches_split_steps_at_level_values():
    # the table/digit path of the symmetric chain equals the continuous symmetric steps
    # evaluated at the quantised coefficients
    rng = np.random.default_rng(12)
    n = 2
    H0 = inputs.drift_zz(n, rng.uniform(-5e3, 5e3, n), np.array([[0, 120.0], [0, 0]]))
    Hk = inputs.controls_global_xy(n)
    lo, hi, L, b, d, dt = np.array([-6e4, -6e4]), np.array([6e4, 6e4]), 4096, 64, 2, 1e-6
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, b, d)
    Dh = O.half_drift(H0, dt)
    assert np.abs(Dh @ Dh - D).max() < 1e-14
    u = rng.uniform(-6e4, 6e4, size=(1, 12, 2))
    q, _, _ = O.quantize(u, lo, hi, L)
    dig = O.level_digits(q, b, d)
    U = O.propagate_strang(T, Dh, dig[0])
    ref = np.eye(4, dtype=complex)
    for row in O.level_values(q[0], lo, hi, L):
        ref = O.strang_split_step(H0, Hk, dt, row) @ ref
    assert np.abs(U - ref).max() < 1e-12
    ex, X = O.simulate_expectation_strang(T, Dh, dig[0], np.eye(4)[0].astype(complex), np.array([1., 1., -1., -1.]))
    assert np.abs(X - U).max() < 1e-15 and ex[0] == 1.0


def test_strang_expectation_series_closed_form_and_prefix_chains():
    # no drift: D_h = I and the symmetric chain is the Rabi rotation at the quantised amplitude,
    # <Z>(t_n) = cos(n dt u_hat) for every n (the whole series, not only its ends)
    H0 = np.zeros((2, 2), dtype=complex)
    Hk = np.stack([SX / 2])
    lo, hi, L, b, d, dt = np.array([-6e4]), np.array([6e4]), 4096, 64, 2, 1e-6
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, b, d)
    Dh = O.half_drift(H0, dt)
    M = 40
    q, _, _ = O.quantize(np.full((1, M, 1), 3.3e4), lo, hi, L)
    uh = O.level_values(q[0, 0], lo, hi, L)[0]
    ex, _ = O.simulate_expectation_strang(T, Dh, O.level_digits(q, b, d)[0], np.array([1, 0], dtype=complex),
                                          np.array([1.0, -1.0]))
    assert np.abs(ex - np.cos(np.arange(M + 1) * dt * uh)).max() < 1e-12
    # with a drift: <O>(t_n) is the expectation in the state of the first n symmetric steps
    rng = np.random.default_rng(14)
    n = 2
    H0 = inputs.drift_zz(n, rng.uniform(-5e3, 5e3, n), np.array([[0, 150.0], [0, 0]]))
    Hk = inputs.controls_global_xy(n)
    lo2, hi2 = np.array([-6e4, -6e4]), np.array([6e4, 6e4])
    T, D = O.build_table(H0, Hk, dt, lo2, hi2, L, b, d)
    Dh = O.half_drift(H0, dt)
    q, _, _ = O.quantize(rng.uniform(-6e4, 6e4, size=(1, 9, 2)), lo2, hi2, L)
    dig = O.level_digits(q, b, d)[0]
    psi0 = np.array([0.6, 0.8j, 0, 0], dtype=complex)
    obs = np.array([1.0, 0.3, -0.5, -1.0])
    ex, _ = O.simulate_expectation_strang(T, Dh, dig, psi0, obs)
    for m in range(10):
        psi = O.propagate_strang(T, Dh, dig[:m]) @ psi0
        assert abs(ex[m] - float(np.sum(obs * np.abs(psi) ** 2))) < 1e-13


def test_strang_commuting_case_has_no_splitting_error():
    n = 2
    rng = np.random.default_rng(13)
    H0 = inputs.drift_zz(n, rng.uniform(-5e3, 5e3, n), np.array([[0, 150.0], [0, 0]]))
    Hk = np.stack([inputs.embed({0: SZ / 2}, n), inputs.embed({1: SZ / 2}, n)])
    lo, hi, L, b, d, dt = np.array([-6e4, -6e4]), np.array([6e4, 6e4]), 4096, 64, 2, 1e-6
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, b, d)
    u = rng.uniform(-6e4, 6e4, size=(1, 20, 2))
    q, _, _ = O.quantize(u, lo, hi, L)
    U = O.propagate_strang(T, O.half_drift(H0, dt, method="eig"), O.level_digits(q, b, d)[0])
    Htot = 20 * H0 + np.tensordot(O.level_values(q[0], lo, hi, L).sum(axis=0), Hk, axes=1)
    assert np.abs(U - O.expm_hermitian(Htot, dt)).max() < 1e-12


def test_chain_time_order():
    # Step 1 is applied first: U = U_2 U_1.  pi/2 about x then pi/2 about y.
    n = 1
    H0 = np.zeros((2, 2), dtype=complex)
    Hk = np.stack([SX / 2, SY / 2])
    dt = 1.0
    L = 3
    lo, hi = np.array([0.0, 0.0]), np.array([math.pi, math.pi])   # levels 0, pi/2, pi
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, L, 1)
    dig = np.array([[[1], [0]], [[0], [1]]])        # step1: x by pi/2; step2: y by pi/2
    U = O.propagate(T, D, dig)
    Rx = O.expm_hermitian(SX / 2, math.pi / 2)
    Ry = O.expm_hermitian(SY / 2, math.pi / 2)
    assert np.abs(U - Ry @ Rx).max() < 1e-15
    assert np.abs(U - Rx @ Ry).max() > 0.1


def test_redo_error_bound_vs_quantization():
    # Per step ||E(u_hat) - E(u)||_2 <= dt |u - u_hat| ||H||_2; the chain error grows at most linearly.
    w = _small_workload(0, M=50)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    U_redo = O.propagate(T, D, dig[0])
    U_split = np.eye(w.N, dtype=complex)
    for n in range(w.M):
        U_split = O.split_step(w.H0, w.Hk, w.dt, w.u[0, n]) @ U_split
    uh = O.level_values(q[0], w.lo, w.hi, w.levels)
    hnorm = [np.linalg.norm(w.Hk[k], 2) for k in range(w.K)]
    bound = sum(w.dt * abs(w.u[0, n, k] - uh[n, k]) * hnorm[k] for n in range(w.M) for k in range(w.K))
    err = np.linalg.norm(U_redo - U_split, 2)
    assert err <= bound * (1 + 1e-9) + 1e-13
    assert err > 0


@pytest.mark.parametrize("n", [1, 3])
def test_fidelity_closed_form_coarse_grain(n):
    # Section II: F = |Tr[e^{i Om dt S} e^{-i Om_hat dt S}]/N|^2; for S = sum X_i/2
    # this is cos^{2n}(dt (Om - Om_hat)/2).
    S = inputs.controls_global_xy(n)[0]
    dt, Om, Omh = 5e-6, 123456.789, 23456.0
    Ua = O.expm_hermitian(S, Om * dt)
    Ub = O.expm_hermitian(S, Omh * dt)
    F = O.fidelity(Ua, Ub)
    assert abs(F - math.cos(dt * (Om - Omh) / 2) ** (2 * n)) < 1e-14
    assert 1 - F > 1e-3


def test_fidelity_invariants():
    rng = np.random.default_rng(7)
    U = inputs.haar_unitary(rng, 8)
    V = inputs.haar_unitary(rng, 8)
    assert abs(O.fidelity(U, U) - 1) < 1e-14
    assert abs(O.fidelity(U, np.exp(0.7j) * U) - 1) < 1e-14
    f = O.fidelity(U, V)
    assert 0 <= f <= 1
    # tau is conjugate-linear in the target, linear in U
    assert abs(O.trace_overlap(U, 1j * V) - 1j * O.trace_overlap(U, V)) < 1e-14
    assert abs(O.trace_overlap(U, V) - np.trace(U.conj().T @ V)) < 1e-13


# ---------------------------------------------------------------- gradient

def _split_fidelity(H0, Hk, dt, u, UT):
    U = np.eye(H0.shape[0], dtype=complex)
    for n in range(u.shape[0]):
        U = O.split_step(H0, Hk, dt, u[n]) @ U
    return O.fidelity(UT, U)


def test_gradient_matches_central_differences():
    w = inputs.config(0, M=8)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    F, g = O.grape_gradient(T, D, w.Hk, w.dt, dig[0], w.target)
    uh = O.level_values(q[0], w.lo, w.hi, w.levels)
    assert abs(F - _split_fidelity(w.H0, w.Hk, w.dt, uh, w.target)) < 1e-13
    Om = w.extra["Omega"]
    h = 1e-6 * Om        # h = 1e-6 in normalised amplitude
    for n in range(w.M):
        for k in range(w.K):
            up, um = uh.copy(), uh.copy()
            up[n, k] += h
            um[n, k] -= h
            fd = (_split_fidelity(w.H0, w.Hk, w.dt, up, w.target)
                  - _split_fidelity(w.H0, w.Hk, w.dt, um, w.target)) / (2 * h)
            assert abs(fd - g[n, k]) < 1e-9 * max(1.0, abs(g).max()) + 2e-12 / h


def test_gradient_single_qubit_closed_form():
    # H0 = 0, control Z/2, target I: F = cos^2(phi/2), phi = dt sum u; dF/du_n = -(dt/2) sin(phi)
    H0 = np.zeros((2, 2), dtype=complex)
    Hk = np.stack([SZ / 2])
    dt, L = 1e-4, 4096
    lo, hi = np.array([-1e4]), np.array([1e4])
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, 64, 2)
    rng = np.random.default_rng(9)
    q, _, _ = O.quantize(rng.uniform(-1e4, 1e4, size=(5, 1)), lo, hi, L)
    dig = O.level_digits(q, 64, 2)
    F, g = O.grape_gradient(T, D, Hk, dt, dig, np.eye(2, dtype=complex))
    phi = dt * O.level_values(q, lo, hi, L).sum()
    assert abs(F - math.cos(phi / 2) ** 2) < 1e-14
    assert np.abs(g[:, 0] + dt / 2 * math.sin(phi)).max() < 1e-16


def _split_state_fidelity(H0, Hk, dt, u, psi0, psiT):
    U = np.eye(H0.shape[0], dtype=complex)
    for n in range(u.shape[0]):
        U = O.split_step(H0, Hk, dt, u[n]) @ U
    return abs(np.conj(psiT) @ U @ psi0) ** 2


def test_state_transfer_gradient_matches_central_differences():
    w = inputs.config(0, M=8)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    rng = np.random.default_rng(21)
    psi0 = np.eye(w.N)[0].astype(complex)
    psiT = rng.normal(size=w.N) + 1j * rng.normal(size=w.N)
    psiT /= np.linalg.norm(psiT)
    F, g = O.state_transfer_gradient(T, D, w.Hk, w.dt, dig[0], psi0, psiT)
    uh = O.level_values(q[0], w.lo, w.hi, w.levels)
    assert abs(F - _split_state_fidelity(w.H0, w.Hk, w.dt, uh, psi0, psiT)) < 1e-13
    h = 1e-6 * w.extra["Omega"]
    for n in range(w.M):
        for k in range(w.K):
            up, um = uh.copy(), uh.copy()
            up[n, k] += h
            um[n, k] -= h
            fd = (_split_state_fidelity(w.H0, w.Hk, w.dt, up, psi0, psiT)
                  - _split_state_fidelity(w.H0, w.Hk, w.dt, um, psi0, psiT)) / (2 * h)
            assert abs(fd - g[n, k]) < 1e-9 * max(1.0, abs(g).max()) + 2e-12 / h


def test_state_transfer_single_qubit_closed_form():
    # H0 = 0, control X/2, |0> -> |1>: F_S = sin^2(phi/2), phi = dt sum u; dF_S/du_n = (dt/2) sin(phi)
    H0 = np.zeros((2, 2), dtype=complex)
    Hk = np.stack([SX / 2])
    dt, L = 1e-4, 4096
    lo, hi = np.array([-1e4]), np.array([1e4])
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, 64, 2)
    rng = np.random.default_rng(22)
    q, _, _ = O.quantize(rng.uniform(-1e4, 1e4, size=(6, 1)), lo, hi, L)
    dig = O.level_digits(q, 64, 2)
    F, g = O.state_transfer_gradient(T, D, Hk, dt, dig, np.array([1, 0], complex), np.array([0, 1], complex))
    phi = dt * O.level_values(q, lo, hi, L).sum()
    assert abs(F - math.sin(phi / 2) ** 2) < 1e-14
    assert np.abs(g[:, 0] - dt / 2 * math.sin(phi)).max() < 1e-16


def test_state_transfer_is_the_unitary_fidelity_of_one_column():
    # for N = 2 and psi_T = U psi0 the state fidelity is 1 and its gradient vanishes
    w = inputs.config(0, n_qubits=1, M=6)
    w.Hk = w.Hk[:2]
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    U = O.propagate(T, D, dig[0])
    psi0 = np.array([0.6, 0.8j])
    F, g = O.state_transfer_gradient(T, D, w.Hk, w.dt, dig[0], psi0, U @ psi0)
    assert abs(F - 1.0) < 1e-14 and np.abs(g).max() < 1e-12


def test_gradient_vanishes_at_reached_target():
    w = inputs.config(0, M=6)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    UT = O.propagate(T, D, dig[0]) * np.exp(0.3j)
    F, g = O.grape_gradient(T, D, w.Hk, w.dt, dig[0], UT)
    assert abs(F - 1) < 1e-13
    assert np.abs(g).max() < 1e-12


# ---------------------------------------------------------------- polar, simulate

def test_polar_factor():
    rng = np.random.default_rng(8)
    U = inputs.haar_unitary(rng, 16)
    assert np.abs(O.polar_unitary(U) - U).max() < 1e-13
    Hp = _rand_herm(rng, 16, 0.01) + np.eye(16)          # positive definite
    P = U @ Hp
    Q = O.polar_unitary(P)
    assert np.abs(Q - U).max() < 1e-12
    assert np.abs(Q.conj().T @ Q - np.eye(16)).max() < 1e-14


def test_expectation_rabi_closed_form():
    # 1 qubit, H0 = 0, constant drive Omega X/2: <Z>(t) = cos(Omega_hat t) exactly.
    H0 = np.zeros((2, 2), dtype=complex)
    Hk = np.stack([SX / 2])
    dt, L, M = 1e-6, 4096, 200
    lo, hi = np.array([0.0]), np.array([2 * 2 * np.pi * 5e3])
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, 64, 2)
    u = np.full((1, M, 1), 2 * np.pi * 5e3 * 1.013)
    q, _, _ = O.quantize(u, lo, hi, L)
    dig = O.level_digits(q, 64, 2)
    psi0 = np.array([1, 0], dtype=complex)
    ex, U = O.simulate_expectation(T, D, dig[0], psi0, np.array([1.0, -1.0]))
    omh = O.level_values(q[0, 0, 0], lo[0], hi[0], L)
    t = dt * np.arange(M + 1)
    assert np.abs(ex - np.cos(omh * t)).max() < 1e-12
    assert ex[0] == 1.0


def _freezing_table(h0, levels_base=100, digits=2, M=400, T=None):
    H0, Hk, rho0, obs = inputs.freezing_system(3, h0)
    T_ = inputs.FREEZE_T if T is None else T
    dt = T_ / M
    lo, hi = np.array([-h0]), np.array([h0])
    Tt, D = O.build_table(H0, Hk, dt, lo, hi, levels_base ** digits, levels_base, digits)
    return H0, Hk, rho0, obs, Tt, D, dt, lo, hi


def test_expect_mixed_zero_drive_closed_form():
    # no drive: the x-magnetisation of the 3-spin Z-Z chain precesses as
    # (2 cos Jt + cos^2 Jt) / 3 (end spins at J, the middle one at 0 or 2J)
    h0 = inputs.FREEZE_H0_AMP
    H0, Hk, rho0, obs, T, D, dt, lo, hi = _freezing_table(h0, levels_base=101, digits=1, M=300, T=6.0)
    q = np.full((1, 300, 1), 50)                        # level 50 of 101 on [-h0, h0] is u = 0
    assert abs(O.level_values(q[0, 0, 0], lo[0], hi[0], 101)) < 1e-12
    ex, _ = O.expect_mixed(T, D, O.level_digits(q, 101, 1)[0], rho0, obs)
    J = h0 / 20.0
    t = dt * np.arange(301)
    Q = ex / ex[0]
    assert ex[0] == 6.0
    assert np.abs(Q - (2 * np.cos(J * t) + np.cos(J * t) ** 2) / 3).max() < 1e-10


def test_expect_mixed_within_quantisation_bound():
    # REDO chain against the unquantised split steps of the same drive: |dQ| <= 3 eps_U with
    # eps_U = sum_n dt |u_n - u^_n| ||H_1||, ||H_1|| = 3/2 (trace norm of rho0 = 6, ||O|| = 3/2)
    h0 = inputs.FREEZE_H0_AMP
    M, Tw = 200, 2 * np.pi
    H0, Hk, rho0, obs, T, D, dt, lo, hi = _freezing_table(h0, M=M, T=Tw)
    u = inputs.freezing_drive([9.0], [0.3], M, h0=h0, T=Tw)
    q, _, _ = O.quantize(u, lo, hi, 10000)
    ex, _ = O.expect_mixed(T, D, O.level_digits(q, 100, 2)[0], rho0, obs)
    X = np.eye(8, dtype=complex)
    ref = [float(np.trace(rho0 @ obs).real)]
    for n in range(M):
        X = O.split_step(H0, Hk, dt, u[0, n]) @ X
        ref.append(float(np.trace(X @ rho0 @ X.conj().T @ obs).real))
    uh = O.level_values(q[0, :, 0], lo[0], hi[0], 10000)
    eps = np.cumsum(dt * np.abs(u[0, :, 0] - uh) * 1.5)
    dQ = np.abs(ex - np.array(ref))[1:] / 6.0
    assert np.all(dQ <= 3 * eps + 1e-12)
    assert dQ.max() > 0                                  # the grid is coarse enough to show


def test_freezing_at_first_bessel_root():
    # Section IV: at lambda = 0 the order parameter reaches ~1 where J0(2 h0 / omega) = 0;
    # the first root is omega_1 = 2 h0 / 2.404825557695773
    h0 = inputs.FREEZE_H0_AMP
    M = 10000
    H0, Hk, rho0, obs, T, D, dt, lo, hi = _freezing_table(h0, M=M)
    w1 = 2 * h0 / 2.404825557695773
    Qbar = {}
    for om in (w1 - 3.0, w1, w1 + 3.0):
        u = inputs.freezing_drive([om], [0.0], M, h0=h0)
        q, _, _ = O.quantize(u, lo, hi, 10000)
        ex, _ = O.expect_mixed(T, D, O.level_digits(q, 100, 2)[0], rho0, obs)
        Qbar[om] = ex[1:].mean() / ex[0]
    assert Qbar[w1] > 0.99
    assert Qbar[w1] > Qbar[w1 - 3.0] + 0.1 and Qbar[w1] > Qbar[w1 + 3.0] + 0.1


# ---------------------------------------------------------------- MLP

def test_gelu_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707
    v = O.gelu(np.array([0.0, 1.0, -1.0, 8.0]))
    assert v[0] == 0.0
    assert abs(v[1] - 0.8413447460685429) < 1e-15
    assert abs(v[2] + 0.15865525393145707) < 1e-15
    assert abs(v[3] - 8.0) < 1e-12


def test_mlp_gradient_finite_difference():
    rng = np.random.default_rng(10)
    params = O.mlp_init([5, 7, 6, 4], rng)
    x = rng.standard_normal((3, 5))
    yt = rng.uniform(-1, 1, size=(3, 4))
    y, cache = O.mlp_forward(params, x)
    loss, grads = O.mlp_backward(params, cache, yt)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[li][0][i, j] += h
            Wm[li][0][i, j] -= h
            lp = np.mean((O.mlp_forward(Wp, x)[0] - yt) ** 2)
            lm = np.mean((O.mlp_forward(Wm, x)[0] - yt) ** 2)
            assert abs((lp - lm) / (2 * h) - grads[li][0][i, j]) < 1e-8
        bp = [(w.copy(), bb.copy()) for w, bb in params]
        bp[li][1][0] += h
        bm = [(w.copy(), bb.copy()) for w, bb in params]
        bm[li][1][0] -= h
        fd = (np.mean((O.mlp_forward(bp, x)[0] - yt) ** 2) - np.mean((O.mlp_forward(bm, x)[0] - yt) ** 2)) / (2 * h)
        assert abs(fd - grads[li][1][0]) < 1e-8


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p2, m, v = O.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p2, p - 0.01 * np.sign(g), atol=1e-7)


# ---------------------------------------------------------------- GRAPE update (Fig. fc)

def test_grape_update_one_step_closed_form():
    # dyadic values: every product and sum below is exact in binary floating point
    u = np.full((2, 3, 2), 0.25)
    g = np.array([0.125, -0.0625])[None, None, :] * np.ones((2, 3, 2))
    lo, hi = np.array([-1.0, -1.0]), np.array([1.0, 1.0])
    out = O.grape_update(u, g, 2.0, np.array([1.0, 0.5]), lo, hi)
    assert np.array_equal(out[0, :, 0], np.full(3, 0.5)) and np.array_equal(out[0, :, 1], np.full(3, 0.125))
    assert np.array_equal(out[1, :, 0], np.full(3, 0.375)) and np.array_equal(out[1, :, 1], np.full(3, 0.1875))
    # no scale means a factor of one for every pulse; the input is left alone
    assert np.array_equal(O.grape_update(u, g, 2.0, None, lo, hi), O.grape_update(u, g, 2.0, np.ones(2), lo, hi))
    assert np.array_equal(u, np.full((2, 3, 2), 0.25))


def test_grape_update_clips_to_each_terms_grid():
    rng = np.random.default_rng(4)
    lo, hi = np.array([-3.0, 0.0, 10.0]), np.array([3.0, 1.0, 20.0])
    u = rng.uniform(lo, hi, size=(4, 50, 3))
    g = rng.standard_normal((4, 50, 3))
    out = O.grape_update(u, g, 1e3, None, lo, hi)           # a huge step lands every entry on an end
    expect = np.where(g > 0, hi[None, None, :], lo[None, None, :])
    assert np.array_equal(out, expect)
    small = O.grape_update(u, g, 1e-3, None, lo, hi)        # a tiny step moves along g, inside the grid
    inside = (u + 1e-3 * g > lo) & (u + 1e-3 * g < hi)
    assert np.array_equal(small[inside], (u + 1e-3 * g)[inside])


def test_grape_step_scale_schedule():
    s = np.array([1.0, 1.0, 7.5, 2.0])
    assert np.array_equal(O.grape_step_scale(s, np.array([0.1, 0.2, 0.3, 0.4]), None), s)
    out = O.grape_step_scale(s, np.array([0.5, 0.1, 0.9, 0.4]), np.array([0.4, 0.2, 0.8, 0.4]))
    # rose: x1.1; fell: halved; capped at 8; equal counts as not fallen
    assert np.allclose(out, [1.1, 0.5, 8.0, 2.2], rtol=0, atol=1e-15)


def test_grape_adam_first_and_third_step_bias_correction():
    lo, hi = np.array([-10.0]), np.array([10.0])
    b1, b2, eps, lr = 0.9, 0.999, 1e-12, 0.01
    gs = [np.array([[[0.3]], [[-2.0]]]), np.array([[[0.1]], [[-1.0]]]), np.array([[[-0.2]], [[4.0]]])]
    u = np.zeros((2, 1, 1))
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    u1, m, v = O.grape_adam_update(u, gs[0], m, v, 1, lr, lo, hi, b1, b2, eps)
    # step 1: the bias-corrected moments are g and g^2, so the step is lr * g / (|g| + eps)
    assert np.allclose(u1, lr * gs[0] / (np.abs(gs[0]) + eps), rtol=1e-14, atol=0)
    u2, m, v = O.grape_adam_update(u1, gs[1], m, v, 2, lr, lo, hi, b1, b2, eps)
    u3, m, v = O.grape_adam_update(u2, gs[2], m, v, 3, lr, lo, hi, b1, b2, eps)
    # step 3: bias-corrected moments are the normalised exponentially weighted means
    #   m_hat = (b1^2 g1 + b1 g2 + g3) / (1 + b1 + b1^2),  v_hat likewise with b2 and g^2
    g1, g2, g3 = gs
    mh = (b1 ** 2 * g1 + b1 * g2 + g3) / (1 + b1 + b1 ** 2)
    vh = (b2 ** 2 * g1 ** 2 + b2 * g2 ** 2 + g3 ** 2) / (1 + b2 + b2 ** 2)
    assert np.allclose(u3 - u2, lr * mh / (np.sqrt(vh) + eps), rtol=1e-12, atol=0)


def test_grape_adam_constant_gradient_steps_by_lr_and_clips():
    lo, hi = np.array([-0.05]), np.array([0.05])
    u = np.zeros((1, 3, 1))
    g = np.array([1e-7, -3.0, 5e4]).reshape(1, 3, 1)
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    for t in range(1, 8):
        u_prev = u
        u, m, v = O.grape_adam_update(u, g, m, v, t, 0.01, lo, hi)
        # a constant gradient has bias-corrected moments g and g^2 at every step
        expect = np.clip(u_prev + 0.01 * g / (np.abs(g) + 1e-12), -0.05, 0.05)
        assert np.allclose(u, expect, rtol=1e-9, atol=0)
    assert u[0, 1, 0] == -0.05 and u[0, 2, 0] == 0.05


def test_grape_ascent_reaches_a_one_qubit_target():
    # the update ascends the oracle's gradient: a Hadamard-like rotation from a random start
    H0 = 2 * np.pi * 300.0 * SZ / 2
    Hk = np.stack([SX / 2, SY / 2])
    dt, L, M = 1e-5, 4096, 10
    Om = 2 * np.pi * 1e4
    lo, hi = np.array([-Om, -Om]), np.array([Om, Om])
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, 64, 2)
    UT = O.expm_hermitian((SX + SZ) / math.sqrt(2), math.pi / 2)
    u = np.random.default_rng(3).uniform(-Om, Om, size=(1, M, 2)) * 0.3
    scale, F_prev, hist = np.ones(1), None, []
    for _ in range(30):
        q, _, _ = O.quantize(u, lo, hi, L)
        F, g = O.grape_gradient(T, D, Hk, dt, O.level_digits(q, 64, 2)[0], UT)
        hist.append(F)
        scale = O.grape_step_scale(scale, np.array([F]), F_prev)
        F_prev = np.array([F])
        u = O.grape_update(u, g[None], 3e9, scale, lo, hi)
    assert hist[0] < 0.01 and hist[-1] > 0.9999


def _bfgs_inverse(pairs, n):
    """Explicit inverse-Hessian BFGS recursion H <- V^T H V + rho s s^T, V = I - rho y s^T,
    from H0 = gamma I (gamma from the newest pair), as matrices."""
    s, y = pairs[-1]
    H = (s @ y) / (y @ y) * np.eye(n)
    for s, y in pairs:
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def test_lbfgs_two_loop_equals_the_explicit_bfgs_matrix():
    rng = np.random.default_rng(13)
    n = 7
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)                      # f's Hessian (F = -f is concave)
    pairs = []
    for _ in range(4):
        s = rng.standard_normal(n)
        pairs.append((s, A @ s))
        g = rng.standard_normal(n)
        H = _bfgs_inverse(pairs, n)
        assert np.allclose(O.lbfgs_direction(g, pairs), H @ g, rtol=1e-12, atol=1e-12)
    # no pairs: the gradient itself; the newest secant pair is reproduced exactly
    assert np.array_equal(O.lbfgs_direction(g, []), g)
    s, y = pairs[-1]
    assert np.allclose(O.lbfgs_direction(y, pairs), s, rtol=1e-12, atol=1e-12)


def _lbfgs_run(Fg, u0, lo, hi, iters, **kw):
    u, state, hist = u0.copy(), {}, []
    for it in range(iters):
        F, g = Fg(u)
        hist.append(F)
        u, state = O.grape_lbfgs_step(u, g, F, state, lo, hi, first=(it == 0), **kw)
    return state, hist


def test_lbfgs_step_maximises_a_concave_quadratic():
    rng = np.random.default_rng(14)
    M, K = 4, 3
    n = M * K
    A = rng.standard_normal((n, n))
    A = A @ A.T / n + 0.5 * np.eye(n)
    ustar = rng.uniform(-0.5, 0.5, size=(M, K))
    lo, hi = np.full(K, -1.0), np.full(K, 1.0)

    def Fg(u):
        e = (u - ustar).ravel()
        return -0.5 * e @ A @ e, -(A @ e).reshape(M, K)

    state, hist = _lbfgs_run(Fg, np.zeros((M, K)), lo, hi, 60)
    assert np.abs(state["u"] - ustar).max() < 1e-7
    # accepted fidelities never fall
    Fs, u, st = [], np.zeros((M, K)), {}
    for it in range(30):
        F, g = Fg(u)
        u, st = O.grape_lbfgs_step(u, g, F, st, lo, hi, first=(it == 0))
        Fs.append(st["F"])
    assert all(b >= a for a, b in zip(Fs, Fs[1:]))


def test_lbfgs_step_respects_the_grid_and_reaches_a_corner():
    # separable quadratic whose maximiser lies outside the box: the box corner is the answer
    M, K = 3, 2
    lo, hi = np.array([-1.0, -2.0]), np.array([1.0, 2.0])
    ustar = np.tile(np.array([3.0, -5.0]), (M, 1))

    def Fg(u):
        e = u - ustar
        return -0.5 * float(np.sum(e * e)), -e

    state, _ = _lbfgs_run(Fg, np.zeros((M, K)), lo, hi, 40)
    assert np.allclose(state["u"], np.tile(np.array([1.0, -2.0]), (M, 1)), atol=1e-12)


def test_lbfgs_backtracks_and_restarts():
    # a rejected trial halves alpha; after ten halvings the pairs are dropped
    lo, hi = np.array([-10.0]), np.array([10.0])
    u0 = np.zeros((1, 1))
    st = {}
    _, st = O.grape_lbfgs_step(u0, np.array([[1.0]]), 0.0, st, lo, hi, first=True)
    assert st["alpha"] == 1.0 and np.allclose(st["d"], [[0.05 * 10.0]])
    st["pairs"] = [(np.array([1.0]), np.array([1.0]))]
    ut = u0 + st["d"]
    for i in range(1, 11):
        ut, st = O.grape_lbfgs_step(ut, np.array([[1.0]]), -1.0, st, lo, hi)     # F fell: reject
        if i < 10:
            assert st["alpha"] == 0.5 ** i and st["pairs"]
    assert st["alpha"] == 1.0 and st["pairs"] == []


def test_lbfgs_grape_reaches_a_one_qubit_target():
    H0 = 2 * np.pi * 300.0 * SZ / 2
    Hk = np.stack([SX / 2, SY / 2])
    dt, L, M = 1e-5, 4096, 10
    Om = 2 * np.pi * 1e4
    lo, hi = np.array([-Om, -Om]), np.array([Om, Om])
    T, D = O.build_table(H0, Hk, dt, lo, hi, L, 64, 2)
    UT = O.expm_hermitian((SX + SZ) / math.sqrt(2), math.pi / 2)

    def Fg(u):
        q, _, _ = O.quantize(u[None], lo, hi, L)
        return O.grape_gradient(T, D, Hk, dt, O.level_digits(q, 64, 2)[0], UT)

    u0 = np.random.default_rng(3).uniform(-Om, Om, size=(M, 2)) * 0.3
    state, hist = _lbfgs_run(Fg, u0, lo, hi, 30)
    assert hist[0] < 0.01 and state["F"] > 0.9999


# ---------------------------------------------------------------- amplitude/phase controls

def _two_species():
    """Two spin-1/2 species on two qubits: S_x, S_y and the diagonal of S_z for each."""
    Sx = np.stack([np.kron(SX, I2) / 2, np.kron(I2, SX) / 2])
    Sy = np.stack([np.kron(SY, I2) / 2, np.kron(I2, SY) / 2])
    sz = np.stack([np.diag(np.kron(SZ, I2)).real / 2, np.diag(np.kron(I2, SZ)).real / 2])
    return Sx, Sy, sz


def test_phase_rotation_turns_the_x_drive_into_the_xy_drive():
    # Eq. vn: Z (sum A S_x) Z^dag = sum A (S_x cos phi + S_y sin phi); checked through the
    # exponentials against scipy (a Z / Z^dag swap or a sign of phi fails)
    from scipy.linalg import expm
    Sx, Sy, sz = _two_species()
    rng = np.random.default_rng(11)
    for _ in range(5):
        A = rng.uniform(0, 2 * np.pi * 1e4, 2)
        phi = rng.uniform(0, 2 * np.pi, 2)
        dt = 7e-6
        Z = np.diag(O.phase_rotation(phi, sz))
        E = expm(-1j * dt * A[1] * Sx[1]) @ expm(-1j * dt * A[0] * Sx[0])
        H = sum(A[k] * (np.cos(phi[k]) * Sx[k] + np.sin(phi[k]) * Sy[k]) for k in range(2))
        assert np.abs(Z @ E @ Z.conj().T - expm(-1j * dt * H)).max() < 1e-13


def test_phase_step_at_levels_matches_the_xy_exponential():
    # table form at the quantised amplitudes = exp(-i dt sum A_hat (S_x cos phi + S_y sin phi)) D,
    # drift first in time
    from scipy.linalg import expm
    Sx, Sy, sz = _two_species()
    rng = np.random.default_rng(12)
    H0 = np.diag(rng.uniform(-3e4, 3e4, 4)).astype(complex)
    dt, base, digits = 2e-6, 16, 2
    levels = base ** digits
    lo, hi = np.zeros(2), np.full(2, 2 * np.pi * 1e4)
    T, D = O.build_table(H0, Sx, dt, lo, hi, levels, base, digits)
    amp = rng.uniform(0, hi[0], (6, 2))
    phi = rng.uniform(0, 2 * np.pi, (6, 2))
    q, _, _ = O.quantize(amp[None], lo, hi, levels)
    dig = O.level_digits(q, base, digits)[0]
    ahat = O.level_values(q[0], lo, hi, levels)
    for n in range(6):
        H = sum(ahat[n, k] * (np.cos(phi[n, k]) * Sx[k] + np.sin(phi[n, k]) * Sy[k]) for k in range(2))
        ref = expm(-1j * dt * H) @ expm(-1j * dt * H0)
        assert np.abs(O.phase_step_propagator(T, D, dig[n], phi[n], sz) - ref).max() < 1e-12
    # the continuous form at the level values is the same operator
    assert np.abs(O.phase_split_step(H0, Sx, sz, dt, ahat[2], phi[2])
                  - O.phase_step_propagator(T, D, dig[2], phi[2], sz)).max() < 1e-12


def test_phase_zero_is_the_x_only_chain():
    Sx, _, sz = _two_species()
    rng = np.random.default_rng(13)
    H0 = np.diag(rng.uniform(-3e4, 3e4, 4)).astype(complex)
    lo, hi = np.zeros(2), np.full(2, 2 * np.pi * 1e4)
    T, D = O.build_table(H0, Sx, 1e-6, lo, hi, 256, 16, 2)
    q, _, _ = O.quantize(rng.uniform(0, hi[0], (1, 9, 2)), lo, hi, 256)
    dig = O.level_digits(q, 16, 2)[0]
    U0 = O.propagate_phase(T, D, dig, np.zeros((9, 2)), sz)
    assert np.abs(U0 - O.propagate(T, D, dig)).max() < 1e-15
    # a phase common to the whole pulse conjugates the x-only chain by Z only if the drift
    # commutes with S_z (it does: diagonal); a phase of pi flips the sign of the drive
    U1 = O.propagate_phase(T, D, dig, np.full((9, 2), np.pi), sz)
    Zpi = np.diag(O.phase_rotation([np.pi, np.pi], sz))
    assert np.abs(U1 - Zpi @ U0 @ Zpi.conj().T).max() < 1e-13


def test_phase_single_spin_closed_form():
    # one spin, no drift, constant amplitude on the grid and phase phi for M steps:
    # U = cos(A T / 2) I - i sin(A T / 2) (cos phi X + sin phi Y)
    base, digits = 16, 2
    levels = base ** digits
    lo, hi = np.zeros(1), np.array([2 * np.pi * 1e4])
    dt, M = 3e-6, 40
    T, D = O.build_table(np.zeros((2, 2), complex), (SX / 2)[None], dt, lo, hi, levels, base, digits)
    qv = 173
    A = lo[0] + qv * (hi[0] - lo[0]) / (levels - 1)
    dig = O.level_digits(np.full((M, 1), qv), base, digits)
    for phi in (0.0, 0.4, 2.5, -1.1):
        U = O.propagate_phase(T, D, dig, np.full((M, 1), phi), (np.diag(SZ).real / 2)[None])
        th = A * M * dt / 2
        ref = np.cos(th) * I2 - 1j * np.sin(th) * (np.cos(phi) * SX + np.sin(phi) * SY)
        assert np.abs(U - ref).max() < 1e-12


def _phase_system(seed=21, M=5):
    Sx, Sy, sz = _two_species()
    rng = np.random.default_rng(seed)
    H0 = np.diag(rng.uniform(-3e4, 3e4, 4)).astype(complex)
    dt, base, digits = 2e-6, 16, 2
    lo, hi = np.zeros(2), np.full(2, 2 * np.pi * 2e4)
    T, D = O.build_table(H0, Sx, dt, lo, hi, base ** digits, base, digits)
    q, _, _ = O.quantize(rng.uniform(0, hi[0], (1, M, 2)), lo, hi, base ** digits)
    dig = O.level_digits(q, base, digits)[0]
    ahat = O.level_values(q[0], lo, hi, base ** digits)
    phi = rng.uniform(0, 2 * np.pi, (M, 2))
    from scipy.stats import unitary_group
    UT = unitary_group.rvs(4, random_state=seed)
    return H0, Sx, Sy, sz, dt, T, D, dig, ahat, phi, UT


def test_phase_gradient_matches_central_differences():
    # derivatives of F of the continuous amplitude/phase chain (Pade exponentials, unquantised
    # amplitudes at the level values) by central differences in A_kn and phi_kn
    H0, Sx, Sy, sz, dt, T, D, dig, ahat, phi, UT = _phase_system()
    F, gA, gphi = O.phase_gradient(T, D, Sx, sz, dt, dig, phi, UT)

    def fid(a, p):
        U = np.eye(4, dtype=complex)
        for n in range(a.shape[0]):
            U = O.phase_split_step(H0, Sx, sz, dt, a[n], p[n]) @ U
        return O.fidelity(UT, U)
    assert abs(F - fid(ahat, phi)) < 1e-12
    for n in range(phi.shape[0]):
        for k in range(2):
            h = 10.0                                     # rad/s: dt h = 2e-5 rad
            ap, am = ahat.copy(), ahat.copy()
            ap[n, k] += h
            am[n, k] -= h
            assert abs((fid(ap, phi) - fid(am, phi)) / (2 * h) - gA[n, k]) <= 1e-7 * np.abs(gA).max()
            e = 1e-5
            pp, pm = phi.copy(), phi.copy()
            pp[n, k] += e
            pm[n, k] -= e
            assert abs((fid(ahat, pp) - fid(ahat, pm)) / (2 * e) - gphi[n, k]) <= 1e-7 * np.abs(gphi).max()


def test_phase_gradient_zero_phase_amplitudes_are_the_x_gradient():
    H0, Sx, Sy, sz, dt, T, D, dig, ahat, phi, UT = _phase_system(22)
    F, gA, _ = O.phase_gradient(T, D, Sx, sz, dt, dig, np.zeros_like(phi), UT)
    Fo, go = O.grape_gradient(T, D, Sx, dt, dig, UT)
    assert abs(F - Fo) < 1e-14 and np.abs(gA - go).max() <= 1e-12 * np.abs(go).max()


def test_phase_gradient_single_spin_common_axis_closed_form():
    # one spin, no drift, every step with the same amplitude A (on the grid) and phase phi: the
    # steps commute, U = exp(-i theta (cos phi X + sin phi Y)/2), theta = A M dt; against the
    # target exp(-i theta_T X / 2), tau = 2 cos(theta_T/2) cos(theta/2) + 2 sin(theta_T/2) sin(theta/2) cos phi,
    # and the step derivatives add up to the derivatives in the common A and phi
    base, digits = 16, 2
    levels = base ** digits
    lo, hi = np.zeros(1), np.array([2 * np.pi * 1e4])
    dt, M = 3e-6, 12
    T, D = O.build_table(np.zeros((2, 2), complex), (SX / 2)[None], dt, lo, hi, levels, base, digits)
    qv = 201
    A = lo[0] + qv * (hi[0] - lo[0]) / (levels - 1)
    dig = O.level_digits(np.full((M, 1), qv), base, digits)
    thT, phi = 0.7, 0.9
    UT = np.cos(thT / 2) * I2 - 1j * np.sin(thT / 2) * SX
    F, gA, gphi = O.phase_gradient(T, D, (SX / 2)[None], (np.diag(SZ).real / 2)[None], dt, dig,
                                   np.full((M, 1), phi), UT)
    th = A * M * dt
    tau = 2 * np.cos(thT / 2) * np.cos(th / 2) + 2 * np.sin(thT / 2) * np.sin(th / 2) * np.cos(phi)
    assert abs(F - tau * tau / 4) < 1e-13
    dtau_dth = -np.cos(thT / 2) * np.sin(th / 2) + np.sin(thT / 2) * np.cos(th / 2) * np.cos(phi)
    dtau_dphi = -2 * np.sin(thT / 2) * np.sin(th / 2) * np.sin(phi)
    assert abs(gA.sum() - 2 * tau * dtau_dth * M * dt / 4) < 1e-12 * abs(gA.sum()) + 1e-15
    assert abs(gphi.sum() - 2 * tau * dtau_dphi / 4) < 1e-12
