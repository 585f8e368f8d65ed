"""The seeded input generators shared by the CUDA path and the oracle (CPU only).

They hold none of the method's arithmetic, but every parity case and the benchmark stand on
them, so the recipe is checked against what fixes it independently: the Haar measure by a
moment it must reproduce, the Ornstein-Uhlenbeck process by its stationary variance and
correlation, the qubit order and the drift by a Kronecker-product construction, and the
workload shapes by the sizes they are built for.
"""
import numpy as np
import pytest

from paper_1707_02162_gb300 import inputs

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)


def _kron_list(ops):
    out = np.ones((1, 1), dtype=complex)
    for op in ops:
        out = np.kron(out, op)
    return out


def test_haar_unitary_is_unitary_and_reproduces_the_trace_moment():
    # for Haar-distributed U(N), E|Tr U|^2 = 1 and E Tr U = 0; dropping the phase fix of
    # the QR factor biases both (the diagonal of R is then positive)
    rng = np.random.default_rng(0)
    N, S = 4, 6000
    tr = np.empty(S, dtype=complex)
    for s in range(S):
        U = inputs.haar_unitary(rng, N)
        if s < 20:
            assert np.abs(U.conj().T @ U - np.eye(N)).max() < 1e-13
        tr[s] = np.trace(U)
    assert abs(np.mean(np.abs(tr) ** 2) - 1.0) < 0.08       # std of the mean ~0.013
    assert abs(np.mean(tr)) < 0.06


def test_ou_noise_stationary_variance_and_correlation():
    rng = np.random.default_rng(1)
    sigma, tau, dt = 0.1, 50e-6, 1e-6
    xi = inputs.ou_noise(rng, 4000, 120, sigma, tau, dt)
    a = np.exp(-dt / tau)
    var = np.mean(xi ** 2, axis=0)                            # per step over realisations
    assert np.all(np.abs(var / sigma ** 2 - 1.0) < 0.1)       # stationary from the first step
    assert abs(np.mean(var) / sigma ** 2 - 1.0) < 0.03
    c1 = np.mean(xi[:, 1:] * xi[:, :-1]) / np.mean(xi ** 2)
    assert abs(c1 - a) < 0.005
    c10 = np.mean(xi[:, 10:] * xi[:, :-10]) / np.mean(xi ** 2)
    assert abs(c10 - a ** 10) < 0.02
    assert abs(np.mean(xi)) < 0.01 * sigma * 10


def test_drift_matches_the_kronecker_construction_with_qubit_zero_first():
    n = 3
    rng = np.random.default_rng(2)
    nu = rng.uniform(-5e3, 5e3, n)
    J = np.triu(rng.uniform(-200, 200, (n, n)), 1)
    ref = np.zeros((8, 8), dtype=complex)
    for i in range(n):
        ops = [I2] * n
        ops[i] = Z / 2
        ref += 2 * np.pi * nu[i] * _kron_list(ops)
        for j in range(i + 1, n):
            ops = [I2] * n
            ops[i] = Z
            ops[j] = Z
            ref += 2 * np.pi * J[i, j] * _kron_list(ops) / 4
    H0 = inputs.drift_zz(n, nu, J)
    assert np.abs(H0 - ref).max() < 1e-9
    # basis index 0b100: qubit 0 (the most significant bit) is down
    assert np.isclose(H0[4, 4].real,
                      np.pi * (-nu[0] + nu[1] + nu[2]) + np.pi / 2 * (-J[0, 1] - J[0, 2] + J[1, 2]))


def test_control_order_and_spin_algebra():
    n = 2
    Hk = inputs.controls_local_xy(n)
    assert Hk.shape == (4, 4, 4)
    assert np.allclose(Hk[0], np.kron(X / 2, I2)) and np.allclose(Hk[1], np.kron(Y / 2, I2))
    assert np.allclose(Hk[2], np.kron(I2, X / 2)) and np.allclose(Hk[3], np.kron(I2, Y / 2))
    # [X/2, Y/2] = i Z/2 on the same qubit, and different qubits commute
    assert np.allclose(Hk[0] @ Hk[1] - Hk[1] @ Hk[0], 1j * np.kron(Z / 2, I2))
    assert np.allclose(Hk[0] @ Hk[3], Hk[3] @ Hk[0])
    g = inputs.controls_global_xy(n)
    assert np.allclose(g[0], Hk[0] + Hk[2]) and np.allclose(g[1], Hk[1] + Hk[3])
    assert np.allclose(inputs.controls_global_x(n)[0], g[0])
    assert np.allclose(inputs.pauli_string("XZ"), np.kron(X, Z))


@pytest.mark.parametrize("idx,n,K,B,M,dt", [(0, 3, 2, 1, 1000, 1e-6), (1, 6, 12, 256, 2000, 1e-6),
                                             (2, 8, 16, 1, 1000, 2e-6), (3, 10, 1, 64, 2000, 1e-6),
                                             (4, 5, 10, 1, 500, 2e-6)])
def test_workload_shapes(idx, n, K, B, M, dt):
    # the sizes each workload is built for; N=1024 is checked without its 2000-step pulses
    w = inputs.config(idx, M=(M if idx != 3 else 8))
    assert w.N == 2 ** n and w.K == K and w.B == B and w.dt == dt
    if idx != 3:
        assert w.M == M
    assert w.levels == 4096 and w.base == 64 and w.digits == 2
    assert np.allclose(w.H0, w.H0.conj().T) and all(np.allclose(h, h.conj().T) for h in w.Hk)
    Om = w.extra["Omega"]
    if idx == 3:
        assert np.allclose(w.lo, 0.0) and np.allclose(w.hi, 2 * Om)
        assert w.psi0[0] == 1.0 and np.sum(np.abs(w.psi0)) == 1.0
        assert w.obs_diag[0] == 1.0 and w.obs_diag[-1] == -1.0 and w.obs_diag[2 ** (n - 1)] == -1.0
    else:
        assert np.allclose(w.lo, -Om) and np.allclose(w.hi, Om)
        assert np.all(np.abs(w.u) <= Om)


def test_workloads_are_deterministic_by_seed():
    a = inputs.config(1, B=2, M=3)
    b = inputs.config(1, B=2, M=3)
    c = inputs.config(1, B=2, M=3, seed=2)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.H0, b.H0) and np.array_equal(a.target, b.target)
    assert not np.array_equal(a.u, c.u)


def test_warm_start_instances_and_drift_diagonals():
    w = inputs.config(4, B=3, M=5)
    assert w.extra["nu"].shape == (3, 5) and w.extra["J"].shape == (3, 5, 5)
    assert len(w.extra["strings"]) == 8 and "IIIII" not in w.extra["strings"]
    assert len(set(w.extra["strings"])) == 8
    h = inputs.drift_diagonals(w)
    for b in range(3):
        assert np.allclose(h[b], np.diag(inputs.drift_zz(5, w.extra["nu"][b], w.extra["J"][b])).real)
    G = inputs.pauli_generator(w.extra["strings"], w.extra["theta"][0])
    assert np.allclose(G, G.conj().T)


def test_phase_workload_species_diagonals():
    w = inputs.phase_config(3, B=2, M=4)
    sz = w.extra["sz"]
    for i in range(3):
        ops = [I2] * 3
        ops[i] = Z / 2
        assert np.allclose(sz[i], np.diag(_kron_list(ops)).real)
    assert np.all((w.u >= 0) & (w.u <= w.extra["Omega"]))
    assert np.all((w.extra["phi"] >= 0) & (w.extra["phi"] < 2 * np.pi))


def test_freezing_drive_and_system():
    M, h0 = 64, inputs.FREEZE_H0_AMP
    om, la = np.array([1.5, 4.0]), np.array([0.0, 1.0])
    u = inputs.freezing_drive(om, la, M)
    assert u.shape == (4, M, 1)
    t = (np.arange(M) + 0.5) * inputs.FREEZE_T / M
    assert np.allclose(u[0, :, 0], h0 * np.cos(1.5 * t))          # omega-major, lambda = 0
    assert np.allclose(u[2, :, 0], h0 * np.cos(4.0 * t))
    assert np.all(np.abs(u[1, :, 0]) <= h0) and np.all(np.abs(u[3, :, 0]) <= h0)
    H0, Hk, rho0, obs = inputs.freezing_system(3)
    Hx, Hkx, rx, ox = inputs.freezing_system(3, basis="x")
    Hd = _kron_list([np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)] * 3)
    assert np.allclose(Hx, Hd @ H0 @ Hd) and np.allclose(Hkx[0], Hd @ Hk[0] @ Hd)
    assert np.allclose(np.diag(rx), Hd @ rho0 @ Hd) and np.allclose(rx, ox)
