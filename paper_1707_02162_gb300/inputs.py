"""Seeded synthetic inputs for the REDO workloads (problem statement only).

This module builds the *inputs* of the REDO problem -- spin Hamiltonians,
control operators, bounded piecewise-constant control amplitudes, target
unitaries and drive noise -- for the five workload shapes used by the tests and
the benchmark.  It holds none of the method's arithmetic (no quantizer, no
exponential, no operator product, no fidelity): both the CUDA path and the CPU
oracle receive the arrays built here.

Conventions
-----------
* Qubit 0 is the most significant bit of the basis index (``np.kron`` order).
* Spin-1/2 operators are Pauli/2; Hamiltonians are in rad/s, time in seconds.
* The drift follows the NMR form of Section III: resonance offsets plus
  Z-Z couplings, ``H0 = sum_i 2 pi nu_i Z_i/2 + sum_{i<j} 2 pi J_ij Z_i Z_j/4``.
* Controls are x/y spin operators (Eq. vn with phases 0 and pi/2).
* Random draws use ``numpy.random.default_rng(seed)`` (PCG64) in the order:
  offsets nu, couplings J (i<j lexicographic), targets, pulses, noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": _I2, "X": _X, "Y": _Y, "Z": _Z}


def embed(ops: dict[int, np.ndarray], n: int) -> np.ndarray:
    """Tensor product with ``ops[i]`` on qubit i and identity elsewhere."""
    out = np.ones((1, 1), dtype=np.complex128)
    for i in range(n):
        out = np.kron(out, ops.get(i, _I2))
    return out


def pauli_string(s: str) -> np.ndarray:
    """Matrix of a Pauli string such as ``"XIZY"`` (character i acts on qubit i)."""
    return embed({i: PAULI[c] for i, c in enumerate(s)}, len(s))


def drift_zz(n: int, nu_hz: np.ndarray, J_hz: np.ndarray) -> np.ndarray:
    """``H0 = sum_i 2pi nu_i Z_i/2 + sum_{i<j} 2pi J_ij Z_i Z_j/4`` (diagonal).

    ``J_hz`` is an (n, n) array; only entries i<j are read.
    """
    N = 2 ** n
    h = np.zeros(N, dtype=np.float64)
    idx = np.arange(N)
    # z_i(a) = +1 if bit of qubit i (MSB first) is 0, else -1
    z = np.stack([1.0 - 2.0 * ((idx >> (n - 1 - i)) & 1) for i in range(n)])
    for i in range(n):
        h += 2.0 * np.pi * nu_hz[i] * z[i] / 2.0
    for i in range(n):
        for j in range(i + 1, n):
            if J_hz[i, j] != 0.0:
                h += 2.0 * np.pi * J_hz[i, j] * z[i] * z[j] / 4.0
    return np.diag(h).astype(np.complex128)


def controls_global_xy(n: int) -> np.ndarray:
    """Two global controls ``sum_i X_i/2`` and ``sum_i Y_i/2``: shape (2, N, N)."""
    hx = sum(embed({i: _X / 2}, n) for i in range(n))
    hy = sum(embed({i: _Y / 2}, n) for i in range(n))
    return np.stack([hx, hy])


def controls_local_xy(n: int) -> np.ndarray:
    """Per-qubit controls ordered X_0/2, Y_0/2, X_1/2, Y_1/2, ...: shape (2n, N, N)."""
    ops = []
    for i in range(n):
        ops.append(embed({i: _X / 2}, n))
        ops.append(embed({i: _Y / 2}, n))
    return np.stack(ops)


def controls_global_x(n: int) -> np.ndarray:
    """One global control ``sum_i X_i/2``: shape (1, N, N)."""
    return np.stack([sum(embed({i: _X / 2}, n) for i in range(n))])


def haar_unitary(rng: np.random.Generator, N: int) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of
    diag(R) moved into Q (Mezzadri 2007)."""
    Zm = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Zm)
    d = np.diagonal(R)
    return Q * (d / np.abs(d))[None, :]


def ou_noise(rng: np.random.Generator, B: int, M: int, sigma: float, tau: float, dt: float) -> np.ndarray:
    """Stationary Ornstein-Uhlenbeck samples xi[B][M]: xi_0 ~ N(0, sigma^2),
    xi_{n+1} = a xi_n + sigma sqrt(1-a^2) z_n with a = exp(-dt/tau) (exact update)."""
    a = np.exp(-dt / tau)
    s = sigma * np.sqrt(1.0 - a * a)
    xi = np.empty((B, M), dtype=np.float64)
    xi[:, 0] = sigma * rng.standard_normal(B)
    z = rng.standard_normal((B, M - 1))
    for n in range(1, M):
        xi[:, n] = a * xi[:, n - 1] + s * z[:, n - 1]
    return xi


@dataclass
class Workload:
    """One REDO problem instance (or a batch of pulses on one system)."""

    name: str
    n_qubits: int
    H0: np.ndarray            # (N, N) complex128, Hermitian drift
    Hk: np.ndarray            # (K, N, N) complex128, Hermitian control terms
    dt: float                 # seconds
    lo: np.ndarray            # (K,) lower end of each coefficient's level grid
    hi: np.ndarray            # (K,) upper end
    levels: int               # L = base**digits
    base: int
    digits: int
    u: np.ndarray             # (B, M, K) float64 control coefficients, rad/s
    target: np.ndarray | None = None   # (N, N) or (B, N, N) complex128
    psi0: np.ndarray | None = None     # (N,) complex128
    obs_diag: np.ndarray | None = None # (N,) float64 diagonal observable
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.H0.shape[0]

    @property
    def K(self) -> int:
        return self.Hk.shape[0]

    @property
    def B(self) -> int:
        return self.u.shape[0]

    @property
    def M(self) -> int:
        return self.u.shape[1]


def _offsets_couplings(rng, n, nu_khz=5.0, J_hz=200.0, chain_only=False):
    nu = rng.uniform(-nu_khz * 1e3, nu_khz * 1e3, size=n)
    J = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if chain_only and j != i + 1:
                continue
            J[i, j] = rng.uniform(-J_hz, J_hz)
    return nu, J


def config(idx: int, *, B: int | None = None, M: int | None = None, n_qubits: int | None = None,
           seed: int | None = None, base: int = 64, digits: int = 2) -> Workload:
    """The five workload shapes (indices 0-4), optionally shrunk for tests.

    0: n=3 (N=8), global X/Y controls, M=1000, dt=1us, B=1, Haar target.
    1: n=6 (N=64), per-qubit X/Y controls (K=12), B=256, M=2000, dt=1us.
    2: n=8 (N=256), K=16, M=1000, dt=2us, B=1, Haar target (GRAPE).
    3: n=10 (N=1024), ZZ chain, K=1 global X with Omega(1+xi(t)), OU noise,
       B=64 realisations, M=2000, dt=1us, psi0=|0..0>, observable Z on qubit 0.
    4: n=5 (N=32), K=10, M=500, dt=2us, targets exp(-i sum theta_k P_k).
    Amplitudes are uniform on [-Omega, Omega] (Omega = 2 pi 10 kHz) except in 3.
    """
    seed = idx if seed is None else seed
    rng = np.random.default_rng(seed)
    L = base ** digits
    if idx == 0:
        n = 3 if n_qubits is None else n_qubits
        B = 1 if B is None else B
        M = 1000 if M is None else M
        Om = 2 * np.pi * 1e4
        nu, J = _offsets_couplings(rng, n)
        H0 = drift_zz(n, nu, J)
        Hk = controls_global_xy(n)
        target = haar_unitary(rng, 2 ** n)
        u = rng.uniform(-Om, Om, size=(B, M, Hk.shape[0]))
        return Workload("plain_redo_n3", n, H0, Hk, 1e-6, np.full(2, -Om), np.full(2, Om), L, base,
                        digits, u, target=target, extra={"Omega": Om})
    if idx == 1:
        n = 6 if n_qubits is None else n_qubits
        B = 256 if B is None else B
        M = 2000 if M is None else M
        Om = 2 * np.pi * 1e4
        nu, J = _offsets_couplings(rng, n)
        H0 = drift_zz(n, nu, J)
        Hk = controls_local_xy(n)
        target = haar_unitary(rng, 2 ** n)
        u = rng.uniform(-Om, Om, size=(B, M, Hk.shape[0]))
        K = Hk.shape[0]
        return Workload("batched_prop_n6", n, H0, Hk, 1e-6, np.full(K, -Om), np.full(K, Om), L, base,
                        digits, u, target=target, extra={"Omega": Om})
    if idx == 2:
        n = 8 if n_qubits is None else n_qubits
        B = 1 if B is None else B
        M = 1000 if M is None else M
        Om = 2 * np.pi * 1e4
        nu, J = _offsets_couplings(rng, n)
        H0 = drift_zz(n, nu, J)
        Hk = controls_local_xy(n)
        target = haar_unitary(rng, 2 ** n)
        u = rng.uniform(-Om, Om, size=(B, M, Hk.shape[0]))
        K = Hk.shape[0]
        return Workload("grape_n8", n, H0, Hk, 2e-6, np.full(K, -Om), np.full(K, Om), L, base, digits,
                        u, target=target, extra={"Omega": Om})
    if idx == 3:
        n = 10 if n_qubits is None else n_qubits
        B = 64 if B is None else B
        M = 2000 if M is None else M
        Om = 2 * np.pi * 5e3
        dt = 1e-6
        nu, J = _offsets_couplings(rng, n, chain_only=True)
        H0 = drift_zz(n, nu, J)
        Hk = controls_global_x(n)
        xi = ou_noise(rng, B, M, 0.1, 50e-6, dt)
        u = (Om * (1.0 + xi))[:, :, None]
        N = 2 ** n
        psi0 = np.zeros(N, dtype=np.complex128)
        psi0[0] = 1.0
        idxs = np.arange(N)
        obs = 1.0 - 2.0 * ((idxs >> (n - 1)) & 1).astype(np.float64)
        return Workload("noisy_drive_n10", n, H0, Hk, dt, np.array([0.0]), np.array([2 * Om]), L, base,
                        digits, u, psi0=psi0, obs_diag=obs, extra={"Omega": Om, "xi": xi})
    if idx == 4:
        n = 5 if n_qubits is None else n_qubits
        B = 1 if B is None else B
        M = 500 if M is None else M
        Om = 2 * np.pi * 1e4
        nu = rng.uniform(-5e3, 5e3, size=(B, n))
        Jm = np.zeros((B, n, n))
        for b in range(B):
            for i in range(n):
                for j in range(i + 1, n):
                    Jm[b, i, j] = rng.uniform(-200.0, 200.0)
        strings = []
        while len(strings) < 8:
            s = "".join(rng.choice(list("IXYZ"), size=n))
            if s != "I" * n and s not in strings:
                strings.append(s)
        theta = rng.uniform(0.0, np.pi, size=(B, 8))
        u = rng.uniform(-Om, Om, size=(B, M, 2 * n))
        Hk = controls_local_xy(n)
        K = Hk.shape[0]
        H0 = drift_zz(n, nu[0], Jm[0])
        return Workload("warm_start_n5", n, H0, Hk, 2e-6, np.full(K, -Om), np.full(K, Om), L, base, digits,
                        u, extra={"Omega": Om, "nu": nu, "J": Jm, "strings": strings, "theta": theta})
    raise ValueError(f"unknown workload index {idx}")


def species_z_diagonals(n: int) -> np.ndarray:
    """Diagonals of ``S_z = Z_i/2`` for every qubit i as its own species: shape (n, 2**n)."""
    idx = np.arange(2 ** n)
    return np.stack([(1.0 - 2.0 * ((idx >> (n - 1 - i)) & 1)) / 2.0 for i in range(n)])


def phase_config(n_qubits: int = 6, *, B: int = 256, M: int = 2000, seed: int = 1, base: int = 64,
                 digits: int = 2, dt: float = 1e-6) -> Workload:
    """Amplitude/phase drive (Section III, Eq. vn): every qubit its own species with x-operator
    ``X_i/2`` (``Hk``) and z-operator diagonal ``extra["sz"][i]``; amplitudes uniform on
    [0, Omega] (``u``, levels on [0, Omega]), phases uniform on [0, 2 pi) (``extra["phi"]``,
    shape (B, M, n)), Omega = 2 pi 10 kHz, NMR drift and Haar target as in the x/y workloads.
    The same pulse in x/y form has coefficients ``A cos phi`` and ``A sin phi``."""
    rng = np.random.default_rng(seed)
    n = n_qubits
    Om = 2 * np.pi * 1e4
    nu, J = _offsets_couplings(rng, n)
    H0 = drift_zz(n, nu, J)
    Hk = np.stack([embed({i: _X / 2}, n) for i in range(n)])
    target = haar_unitary(rng, 2 ** n)
    u = rng.uniform(0.0, Om, size=(B, M, n))
    phi = rng.uniform(0.0, 2 * np.pi, size=(B, M, n))
    return Workload(f"amp_phase_n{n}", n, H0, Hk, dt, np.zeros(n), np.full(n, Om), base ** digits, base, digits,
                    u, target=target, extra={"Omega": Om, "phi": phi, "sz": species_z_diagonals(n)})


def drift_diagonals(w: Workload) -> np.ndarray:
    """Each instance's own diagonal drift ``h[b] = diag(H0_b)`` (rad/s), shape (B, N), from the
    per-instance offsets ``extra["nu"]`` and couplings ``extra["J"]`` of the warm-start
    workload (index 4): the input of the per-pulse drift calls, whose table is built with H0 = 0."""
    nu, J = w.extra["nu"], w.extra["J"]
    return np.stack([np.real(np.diag(drift_zz(w.n_qubits, nu[b], J[b]))) for b in range(nu.shape[0])])


def pauli_generator(strings: list[str], theta: np.ndarray) -> np.ndarray:
    """Hermitian generator ``G = sum_k theta_k P_k`` of a target ``exp(-i G)``.

    Only the generator is built here; exponentiating it is left to the caller
    (the target is an input of the control problem, not part of REDO).
    """
    return sum(t * pauli_string(s) for s, t in zip(strings, theta))


# ---------------------------------------------------------------------------
# Noisy exotic freezing (Section IV): driven Ising chain, order parameter Q(omega, lambda)
# ---------------------------------------------------------------------------

FREEZE_H0_AMP = 5 * np.pi        # h0 (rad/s)
FREEZE_T = 20 * np.pi            # averaging window [0, T] (s)


def _hadamard_all(n: int) -> np.ndarray:
    h = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
    out = np.array([[1.0 + 0j]])
    for _ in range(n):
        out = np.kron(out, h)
    return out


def freezing_system(n: int = 3, h0: float = FREEZE_H0_AMP, basis: str = "z"):
    """Ising chain ``H(t) = -J sum_i 2 I_iz I_{i+1,z} - h(t) sum_i I_ix`` with ``J = h0/20``.

    Returns ``(H0, Hk, rho0, obs)``: the drift (the Z-Z chain), one control term
    ``Hk[0] = -sum_i I_ix`` whose coefficient is the drive ``h(t)``, and
    ``rho0 = obs = sum_i I_ix`` (initial deviation density matrix and measured
    x-magnetisation).  ``basis="x"`` conjugates all four by the Hadamard on every
    qubit, where ``rho0`` and ``obs`` become diagonal (returned as their diagonals).
    """
    J = h0 / 20.0
    H0 = -J * sum(2 * embed({i: _Z / 2, i + 1: _Z / 2}, n) for i in range(n - 1))
    Mx = sum(embed({i: _X / 2}, n) for i in range(n))
    Hk = np.stack([-Mx])
    if basis == "z":
        return H0, Hk, Mx.copy(), Mx.copy()
    Hd = _hadamard_all(n)
    rot = lambda A: Hd @ A @ Hd
    m = np.real(np.diag(rot(Mx))).copy()
    return rot(H0), np.stack([rot(Hk[0])]), m, m.copy()


def freezing_drive(omegas: np.ndarray, lams: np.ndarray, M: int, h0: float = FREEZE_H0_AMP,
                   T: float = FREEZE_T, seed: int = 5) -> np.ndarray:
    """Drive coefficients ``h0 {(1 - lambda) cos(omega t_n) + lambda eta_n}`` on M steps of
    ``dt = T/M``, sampled at step midpoints ``t_n = (n + 1/2) dt``, with ``eta_n`` uniform on
    [-1, 1], independent per step and per (omega, lambda) pulse.  Pulses are ordered
    omega-major: pulse ``i * len(lams) + j`` has ``omegas[i]``, ``lams[j]``.  Shape (B, M, 1)."""
    rng = np.random.default_rng(seed)
    omegas = np.asarray(omegas, dtype=np.float64)
    lams = np.asarray(lams, dtype=np.float64)
    dt = T / M
    t = (np.arange(M) + 0.5) * dt
    om = np.repeat(omegas, lams.size)[:, None]
    la = np.tile(lams, omegas.size)[:, None]
    eta = rng.uniform(-1.0, 1.0, size=(om.shape[0], M))
    u = h0 * ((1.0 - la) * np.cos(om * t[None, :]) + la * eta)
    return u[:, :, None]

