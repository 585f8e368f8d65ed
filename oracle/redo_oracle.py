"""CPU FP64 oracle for REDO -- TEST INFRASTRUCTURE ONLY.

Rapid Exponentiation using Discrete Operators (Bhole & Mahesh,
arXiv:1707.02162).  This module is a plain, slow, obviously-correct numpy
restatement of what the GPU library computes.  It exists to check the CUDA
path; nothing in the product imports it.  Only the test-suite, the smoke check
and the benchmark's CPU-baseline arm may call it.  It shares no code with the
CUDA path (no kernels, headers, tables or helpers) and never imports the
product package.

All arithmetic is IEEE float64 / complex128.  Library primitives used as single
steps: matrix product (``@``), ``numpy.linalg.solve`` (Pade denominator),
``numpy.linalg.eigh`` (Hermitian eigen-decomposition).

Functions and the passage each one follows:

* :func:`quantize` / :func:`level_digits` -- Eq. (cgrain), Section II: the
  coefficient is coarse-grained to ``sum_j c_j b^j`` times the grain epsilon.
* :func:`expm_pade13` -- the scaling-and-squaring Pade-13 matrix exponential of
  Higham (2005) ("Pade ME", the paper's comparison method, Section II).
* :func:`expm_hermitian` -- ``exp(-i t H)`` by eigen-decomposition ("ED").
* :func:`build_table` -- the one-time discrete-operator table, process 1 of
  Section II (Eq. redoform, read with the ``c b^j dt`` scaling of the worked
  example that precedes it) plus the drift step ``D = exp(-i dt H0)``.
* :func:`step_factors` / :func:`step_propagator` / :func:`propagate` -- process
  2 (Eq. exp2prod) applied per control term, composed with the drift as in the
  Dirac-frame step of Section III (Eqs. vnd and the step formula after it) and
  chained ``U = U_M ... U_1`` (Section III).
* :func:`fidelity` -- the unitary fidelity ``F_U`` of Section III.
* :func:`grape_gradient` -- the GRAPE gradient ``dF/du_kn`` of the REDO split
  model (Section III, flowchart Fig. fc; the paper gives no formula, the
  derivative is taken from the definitions, see its docstring).
* :func:`state_transfer_gradient` -- the state-to-state fidelity ``|<psi_T|U|psi0>|^2``
  and its GRAPE gradient, from the same definitions.
* :func:`grape_update` / :func:`grape_step_scale` / :func:`grape_adam_update` /
  :func:`lbfgs_direction` / :func:`grape_lbfgs_step` -- the control update of the
  GRAPE loop (Section III, Fig. fc; the rule is this module's reading: clipped ascent
  with per-pulse step factors, Adam, or projected L-BFGS with Armijo backtracking).
* :func:`polar_unitary` -- polar factor ``P (P^dag P)^(-1/2)``.
* :func:`half_drift` / :func:`strang_step_propagator` / :func:`propagate_strang`
  / :func:`strang_split_step` / :func:`simulate_expectation_strang` -- the
  symmetric (Strang) placement of the drift around the control factors of a
  step, the second-order variant of the Section III step.
* :func:`phase_rotation` / :func:`phase_step_propagator` / :func:`propagate_phase` /
  :func:`phase_split_step` / :func:`phase_gradient` -- amplitude/phase controls (Section
  III, Eq. vn and the Dirac-frame step after Eq. vnd): one x-table per species, the phase
  applied as the diagonal rotation Z_n on both sides of the step's control factors; the GRAPE
  gradient in amplitudes and phases from the definitions.
* :func:`simulate_expectation` -- ``<M> = Tr[M rho(t)]`` of Section IV for a
  pure initial state; :func:`expect_mixed` -- the same for a dense (mixed or
  deviation) initial density matrix, the order parameter of the freezing study.
* :func:`mlp_*` -- an FP64 multilayer perceptron with exact (erf) GELU and Adam,
  the learned warm start of the control problem (no counterpart in the paper).

Pins (tests/test_oracle_pins.py) tie every function to closed forms, library
routines used as independent checks (scipy), invariants and brute force.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

__all__ = [
    "quantize", "level_digits", "level_values", "table_thetas", "expm_pade13", "expm_hermitian",
    "build_table", "step_factors", "step_propagator", "propagate", "fidelity", "trace_overlap",
    "grape_gradient", "polar_unitary", "simulate_expectation", "exact_step", "split_step",
    "plan_digits", "grape_update", "grape_step_scale", "grape_adam_update", "lbfgs_direction",
    "grape_lbfgs_step", "mlp_init", "mlp_forward", "mlp_backward", "adam_step", "gelu", "gelu_grad",
]


# ---------------------------------------------------------------------------
# Eq. (cgrain): coarse graining to integer levels
# ---------------------------------------------------------------------------

def quantize(u, lo, hi, levels):
    """Coarse-grain coefficients to level indices (Eq. cgrain, Section II).

    Reading adopted: the grid has ``levels`` points ``lo + q*delta``,
    ``delta = (hi - lo)/(levels - 1)``, both ends included, and a coefficient
    goes to the nearest grid point, ties to even ("floor-ceil" bracket of the
    paper, rounding mode unstated).  Arithmetic: one IEEE subtract, one IEEE
    divide (no fused multiply-add), then round-half-even.

    Returns ``(q, n_nonfinite, n_saturated)``: ``q`` int32 of the shape of u
    (trailing axis = term k), with non-finite inputs mapped to level 0 and
    out-of-range inputs clamped to [0, levels-1].
    """
    u = np.asarray(u, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    delta = (hi - lo) / np.float64(levels - 1)
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        x = np.subtract(u, lo)
        x = np.divide(x, delta)
        r = np.rint(x)
    finite = np.isfinite(u)
    low = finite & (r < 0)
    high = finite & (r > levels - 1)
    r = np.where(low, 0.0, r)
    r = np.where(high, levels - 1, r)
    r = np.where(finite, r, 0.0)
    q = r.astype(np.int32)
    return q, int((~finite).sum()), int(low.sum() + high.sum())


def level_digits(q, base, digits):
    """Base-b digits ``c_j = floor(q / b^j) mod b`` for j = 0..digits-1 (Eq. cgrain).

    The paper's digit range j = l..m maps to 0..digits-1 with the grain
    epsilon = delta, so ``q = sum_j c_j b^j``.  Shape: q.shape + (digits,).
    """
    q = np.asarray(q, dtype=np.int64)
    return np.stack([(q // (base ** j)) % base for j in range(digits)], axis=-1).astype(np.int32)


def level_values(q, lo, hi, levels):
    """Quantised coefficient ``u_hat = lo + q*delta``: the coarse-grained value of Eq. (cgrain),
    Section II."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    delta = (hi - lo) / np.float64(levels - 1)
    return lo + np.asarray(q, dtype=np.float64) * delta


def table_thetas(lo_k, hi_k, levels, base, digits):
    """Coefficients of the discrete operators of one term: ``theta[j][c]``.

    Digit 0 carries the offset of the grid (reading for signed ranges):
    ``theta[0][c] = lo + c*delta``; digit j >= 1: ``theta[j][c] = c * b^j * delta``
    (Eq. redoform read with the ``c b^j`` scaling of the worked example).
    Summing one entry per digit gives ``lo + q*delta`` for ``q = sum_j c_j b^j``.
    """
    delta = (np.float64(hi_k) - np.float64(lo_k)) / np.float64(levels - 1)
    th = np.empty((digits, base), dtype=np.float64)
    for c in range(base):
        th[0, c] = np.float64(lo_k) + np.float64(c) * delta
    for j in range(1, digits):
        for c in range(base):
            th[j, c] = np.float64(c * base ** j) * delta
    return th


def plan_digits(omega_max, eps, base):
    """Cost model of Section II: smallest l with b^l <= eps and m with b^(m+1) > omega_max;
    returns ``(l, m, p, s)`` with ``p = m - l`` products and ``s = (b-1)(p+1)`` stored operators."""
    l = int(math.floor(math.log(eps, base) + 1e-12))
    m = int(math.ceil(math.log(omega_max, base) - 1.0 - 1e-12))
    while base ** (m + 1) <= omega_max:
        m += 1
    p = m - l
    s = (base - 1) * (p + 1)
    return l, m, p, s


# ---------------------------------------------------------------------------
# Matrix exponentials
# ---------------------------------------------------------------------------

def _pade13_coefficients():
    """Coefficients b_j of the [13/13] Pade approximant of exp, the numerator polynomial of
    Higham (2005) for the Pade method the paper compares with (Section II)."""
    # b_j = (26 - j)! 13! / (26! j! (13 - j)!)
    m = 13
    out = []
    for j in range(m + 1):
        f = Fraction(math.factorial(2 * m - j) * math.factorial(m),
                     math.factorial(2 * m) * math.factorial(j) * math.factorial(m - j))
        out.append(float(f))
    return out


_B13 = _pade13_coefficients()
# Higham (2005), Table 2.3: largest 1-norm for which the degree-13 Pade
# approximant meets unit roundoff in double precision.
_THETA13 = 5.371920351148152


def expm_pade13(A):
    """``exp(A)`` by scaling and squaring with the [13/13] Pade approximant (Higham 2005).

    Steps: choose s with ||A/2^s||_1 <= theta_13; evaluate the even/odd parts
    U, V of the approximant at A/2^s; solve (V - U) R = (V + U); square s times.
    """
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    norm1 = np.abs(A).sum(axis=0).max() if n else 0.0
    s = 0
    if norm1 > _THETA13:
        s = int(math.ceil(math.log2(norm1 / _THETA13)))
    A = A / (2.0 ** s)
    I = np.eye(n, dtype=np.complex128)
    A2 = A @ A
    A4 = A2 @ A2
    A6 = A4 @ A2
    b = _B13
    Uin = A6 @ (b[13] * A6 + b[11] * A4 + b[9] * A2) + b[7] * A6 + b[5] * A4 + b[3] * A2 + b[1] * I
    U = A @ Uin
    V = A6 @ (b[12] * A6 + b[10] * A4 + b[8] * A2) + b[6] * A6 + b[4] * A4 + b[2] * A2 + b[0] * I
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


def expm_hermitian(H, t, eig=None):
    """``exp(-i t H)`` for Hermitian H by eigen-decomposition ``H = V diag(w) V^dag`` (the "ED"
    method among the paper's comparison methods, Section II).

    ``eig`` may pass ``(w, V) = numpy.linalg.eigh(H)`` computed once for many ``t``."""
    if eig is None:
        eig = np.linalg.eigh(np.asarray(H, dtype=np.complex128))
    w, V = eig
    return (V * np.exp(-1j * t * w)[None, :]) @ V.conj().T


# ---------------------------------------------------------------------------
# Process 1: the one-time table
# ---------------------------------------------------------------------------

def build_table(H0, Hk, dt, lo, hi, levels, base, digits, method="pade"):
    """Discrete-operator table and drift step (Section II process 1; Section III).

    ``T[k][j][c] = exp(-i dt theta_kjc H_k)`` with ``theta`` from
    :func:`table_thetas`, and ``D = exp(-i dt H0)``.  ``method`` picks the
    exponential: ``"pade"`` (:func:`expm_pade13`) or ``"eig"``
    (:func:`expm_hermitian`).  Returns ``(T, D)`` with T of shape
    (K, digits, base, N, N).  The table is NOT folded with D.
    """
    Hk = np.asarray(Hk, dtype=np.complex128)
    K, N, _ = Hk.shape
    T = np.empty((K, digits, base, N, N), dtype=np.complex128)
    for k in range(K):
        th = table_thetas(lo[k], hi[k], levels, base, digits)
        for j in range(digits):
            for c in range(base):
                if method == "pade":
                    T[k, j, c] = expm_pade13(-1j * dt * th[j, c] * Hk[k])
                else:
                    T[k, j, c] = expm_hermitian(Hk[k], dt * th[j, c])
    if method == "pade":
        D = expm_pade13(-1j * dt * np.asarray(H0, dtype=np.complex128))
    else:
        D = expm_hermitian(H0, dt)
    return T, D


# ---------------------------------------------------------------------------
# Process 2: products of discrete operators, the step and the chain
# ---------------------------------------------------------------------------

def step_factors(T, D, digit_row):
    """Per-term products ``E_k = T[k][d-1][c_{d-1}] ... T[k][0][c_0]`` (Eq. exp2prod).

    ``digit_row`` has shape (K, digits).  Returns the list [E_0, ..., E_{K-1}].
    """
    K, d = digit_row.shape
    out = []
    for k in range(K):
        E = T[k, 0, digit_row[k, 0]]
        for j in range(1, d):
            E = T[k, j, digit_row[k, j]] @ E
        out.append(E)
    return out


def step_propagator(T, D, digit_row):
    """One step ``U_n = E_{K-1} ... E_0 D`` (Section III step formula with the drift
    applied first in time; Lie-Trotter reading of the Dirac-frame product)."""
    U = D
    for E in step_factors(T, D, digit_row):
        U = E @ U
    return U


def propagate(T, D, digits_bm):
    """Chained propagator ``U = U_M ... U_2 U_1`` (Section III) for one pulse.

    ``digits_bm`` has shape (M, K, digits).  Returns the N x N product.
    """
    N = D.shape[0]
    U = np.eye(N, dtype=np.complex128)
    for n in range(digits_bm.shape[0]):
        U = step_propagator(T, D, digits_bm[n]) @ U
    return U


def exact_step(H0, Hk, dt, u_row):
    """Unsplit, unquantised step ``exp(-i dt (H0 + sum_k u_k H_k))`` (Eq. propUn)."""
    H = np.asarray(H0, dtype=np.complex128) + np.tensordot(np.asarray(u_row, dtype=np.float64), Hk, axes=1)
    return expm_pade13(-1j * dt * H)


def split_step(H0, Hk, dt, u_row):
    """Split but unquantised step ``exp(-i dt u_{K-1} H_{K-1}) ... exp(-i dt u_0 H_0) exp(-i dt H0)``:
    the Section III step formula at continuous coefficients (what the table evaluates at the
    quantised ones)."""
    U = expm_pade13(-1j * dt * np.asarray(H0, dtype=np.complex128))
    for k in range(Hk.shape[0]):
        U = expm_pade13(-1j * dt * u_row[k] * Hk[k]) @ U
    return U


# ---------------------------------------------------------------------------
# Symmetric (Strang) splitting -- the second-order variant of the step
# ---------------------------------------------------------------------------
# The step of Section III applies the drift once per step (first order in dt).
# The symmetric variant puts half of it on each side of the control factors:
#     S_n = D_h E_{K-1} ... E_0 D_h,      D_h = exp(-i dt H0 / 2),
# which removes the drift's share of the splitting error: with one control (or
# commuting controls) the one-step error is O(dt^3) instead of O(dt^2); the order
# among non-commuting controls stays that of the Section III step.  Written out
# step by step here, with no use of the identity prod_n S_n = D_h (prod_n E_n D) D_h^dag.

def half_drift(H0, dt, method="pade"):
    """``D_h = exp(-i (dt/2) H0)``: half of the Section III drift step, for the symmetric variant
    of the step that splits the drift evenly around the control factors."""
    if method == "pade":
        return expm_pade13(-0.5j * dt * np.asarray(H0, dtype=np.complex128))
    return expm_hermitian(H0, 0.5 * dt)


def strang_step_propagator(T, Dh, digit_row):
    """One symmetric step ``S_n = D_h E_{K-1} ... E_0 D_h`` (T not folded with the drift): the
    Section III step with the drift split evenly, products of Eq. (exp2prod) as in process 2."""
    U = Dh
    for E in step_factors(T, Dh, digit_row):
        U = E @ U
    return Dh @ U


def propagate_strang(T, Dh, digits_bm):
    """Chained symmetric propagator ``S_M ... S_1`` for one pulse (the Section III chain of
    symmetric steps)."""
    U = np.eye(Dh.shape[0], dtype=np.complex128)
    for n in range(digits_bm.shape[0]):
        U = strang_step_propagator(T, Dh, digits_bm[n]) @ U
    return U


def strang_split_step(H0, Hk, dt, u_row):
    """Symmetric split, unquantised step ``D_h exp(-i dt u_{K-1} H_{K-1}) ... exp(-i dt u_0 H_0) D_h``
    (the Section III step with the drift split evenly, at continuous coefficients)."""
    Dh = expm_pade13(-0.5j * dt * np.asarray(H0, dtype=np.complex128))
    U = Dh
    for k in range(Hk.shape[0]):
        U = expm_pade13(-1j * dt * u_row[k] * Hk[k]) @ U
    return Dh @ U


def simulate_expectation_strang(T, Dh, digits_bm, psi0, obs_diag):
    """``<O>(t_n)`` along the symmetric chain, ``psi_n = S_n ... S_1 psi0`` (Section IV's
    expectation values on the chain of symmetric steps); returns (expect, U_final)."""
    N = Dh.shape[0]
    X = np.eye(N, dtype=np.complex128)
    out = np.empty(digits_bm.shape[0] + 1, dtype=np.float64)
    psi = X @ psi0
    out[0] = float(np.sum(obs_diag * (psi.real ** 2 + psi.imag ** 2)))
    for n in range(digits_bm.shape[0]):
        X = strang_step_propagator(T, Dh, digits_bm[n]) @ X
        psi = X @ psi0
        out[n + 1] = float(np.sum(obs_diag * (psi.real ** 2 + psi.imag ** 2)))
    return out, X


# ---------------------------------------------------------------------------
# Amplitude/phase controls (Section III, Eq. vn and the Dirac-frame step that follows Eq. vnd)
# ---------------------------------------------------------------------------
# A linearly polarised drive on species k, amplitude A_kn and phase phi_kn, is the x-polarised
# drive turned about z:  sum_k A_kn (S_xk cos phi_kn + S_yk sin phi_kn) = Z_n (sum_k A_kn S_xk) Z_n^dag
# with Z_n = exp(-i sum_k phi_kn S_kz).  One x-table per species then serves every phase:
#     U_n = Z_n E_{K-1} ... E_0 Z_n^dag D,
# E_k the table product for the quantised amplitude of species k, drift first in time as in the
# Section III step.  Phases are not quantised: Z_n is diagonal for diagonal S_kz and is evaluated
# per basis state, exp(-i sum_k phi_kn sz[k][a]).

def phase_rotation(phi_row, sz):
    """Diagonal of ``Z_n = exp(-i sum_k phi_kn S_kz)``; ``sz[k]`` is the diagonal of ``S_kz``
    (the phase turn of the drive of Section III, Eq. vn)."""
    return np.exp(-1j * (np.asarray(phi_row, dtype=np.float64) @ np.asarray(sz, dtype=np.float64)))


def phase_step_propagator(T, D, digit_row, phi_row, sz):
    """One amplitude/phase step ``U_n = Z_n E_{K-1} ... E_0 Z_n^dag D`` (T not folded with the drift):
    Section III, Eq. vn and the Dirac-frame step that follows Eq. vnd."""
    Z = np.diag(phase_rotation(phi_row, sz))
    E = np.eye(D.shape[0], dtype=np.complex128)
    for Ek in step_factors(T, D, digit_row):
        E = Ek @ E
    return Z @ E @ Z.conj().T @ D


def propagate_phase(T, D, digits_bm, phi_bm, sz):
    """Chained amplitude/phase propagator ``U_M ... U_1`` for one pulse (Section III);
    ``phi_bm`` is (M, K)."""
    U = np.eye(D.shape[0], dtype=np.complex128)
    for n in range(digits_bm.shape[0]):
        U = phase_step_propagator(T, D, digits_bm[n], phi_bm[n], sz) @ U
    return U


def phase_split_step(H0, Sx, sz, dt, amp_row, phi_row):
    """Unquantised amplitude/phase step ``Z_n exp(-i dt A_{K-1} S_x,K-1) ... exp(-i dt A_0 S_x0) Z_n^dag
    exp(-i dt H0)``: the step of Section III's Eq. vn drive at continuous amplitudes."""
    Z = np.diag(phase_rotation(phi_row, sz))
    E = np.eye(H0.shape[0], dtype=np.complex128)
    for k in range(Sx.shape[0]):
        E = expm_pade13(-1j * dt * amp_row[k] * Sx[k]) @ E
    return Z @ E @ Z.conj().T @ expm_pade13(-1j * dt * np.asarray(H0, dtype=np.complex128))


def phase_gradient(T, D, Sx, sz, dt, digits_bm, phi_bm, U_target):
    """``(F, gA, gphi)``: the unitary fidelity of the amplitude/phase chain and its derivatives
    ``gA[n][k] = dF/dA_kn`` (at the quantised amplitudes) and ``gphi[n][k] = dF/dphi_kn``.

    The paper optimises the control profiles {Omega_kn, phi_kn} by GRAPE (Section III) without
    printing the gradient; this one follows from the definitions.  With ``U = U_M ... U_1``,
    ``X_{n-1} = U_{n-1} ... U_1``, ``L_n = U_M ... U_{n+1}`` and ``tau = Tr(U_T^dag U)``,
    ``dF/dx = (2/N^2) Re(conj(tau) Tr(U_T^dag L_n (dU_n/dx) X_{n-1}))`` for a parameter x of step n,
    where, for ``U_n = Z_n E_{K-1} ... E_0 Z_n^dag D``,
    ``dU_n/dA_kn = Z_n E_{K-1} ... E_{k+1} (-i dt S_xk) E_k ... E_0 Z_n^dag D`` (S_xk commutes with
    its own exponential) and ``dU_n/dphi_kn = -i [S_kz, Z_n E_n Z_n^dag] D``.
    """
    N = D.shape[0]
    M = digits_bm.shape[0]
    K = Sx.shape[0]
    steps = [phase_step_propagator(T, D, digits_bm[n], phi_bm[n], sz) for n in range(M)]
    X = [np.eye(N, dtype=np.complex128)]
    for n in range(M):
        X.append(steps[n] @ X[-1])
    U = X[M]
    L = []                                               # L[n]: the steps after step n (0-based)
    for n in range(M):
        Ln = np.eye(N, dtype=np.complex128)
        for m in range(n + 1, M):
            Ln = steps[m] @ Ln
        L.append(Ln)
    tau = trace_overlap(U_target, U)
    F = (tau.real * tau.real + tau.imag * tau.imag) / float(N * N)
    gA = np.zeros((M, K))
    gphi = np.zeros((M, K))
    Sz = [np.diag(np.asarray(sz[k], dtype=np.float64)).astype(np.complex128) for k in range(K)]
    for n in range(M):
        Z = np.diag(phase_rotation(phi_bm[n], sz))
        E = step_factors(T, D, digits_bm[n])
        Et = np.eye(N, dtype=np.complex128)
        for Ek in E:
            Et = Ek @ Et
        for k in range(K):
            before = np.eye(N, dtype=np.complex128)
            for m in range(k + 1):
                before = E[m] @ before                   # E_k ... E_0
            after = np.eye(N, dtype=np.complex128)
            for m in range(k + 1, K):
                after = E[m] @ after                     # E_{K-1} ... E_{k+1}
            dU = Z @ after @ (-1j * dt * Sx[k]) @ before @ Z.conj().T @ D
            dtau = np.trace(U_target.conj().T @ L[n] @ dU @ X[n])
            gA[n, k] = 2.0 / (N * N) * (np.conj(tau) * dtau).real
            W = Z @ Et @ Z.conj().T
            dU = -1j * (Sz[k] @ W - W @ Sz[k]) @ D
            dtau = np.trace(U_target.conj().T @ L[n] @ dU @ X[n])
            gphi[n, k] = 2.0 / (N * N) * (np.conj(tau) * dtau).real
    return F, gA, gphi


# ---------------------------------------------------------------------------
# Fidelity (Section III, F_U)
# ---------------------------------------------------------------------------

def trace_overlap(U_target, U):
    """``tau = Tr(U_T^dag U) = sum_ab conj(U_T[a,b]) U[a,b]``, the overlap inside the unitary
    fidelity of Section III."""
    return complex(np.sum(np.conj(U_target) * U))


def fidelity(U_target, U):
    """``F_U = |Tr(U_T^dag U)|^2 / N^2`` (``Tr(U_T^dag U_T) = N`` for unitary U_T), the unitary
    fidelity of Section III."""
    N = U.shape[0]
    tau = trace_overlap(U_target, U)
    return (tau.real * tau.real + tau.imag * tau.imag) / float(N * N)


# ---------------------------------------------------------------------------
# GRAPE gradient of the REDO split model
# ---------------------------------------------------------------------------

def grape_gradient(T, D, Hk, dt, digits_bm, U_target):
    """``(F, g)`` with ``g[n][k] = dF/du_kn`` of the split model at the quantised point.

    The paper's GRAPE (Section III, Fig. fc) ascends F with REDO propagators but
    prints no gradient; this one is derived from the definitions.  With
    ``U = U_M ... U_1``, ``X_{n-1} = U_{n-1} ... U_1``, ``L_n = U_M ... U_{n+1}``,
    ``A_k = E_{K-1} ... E_{k+1}`` and ``B_k = E_k ... E_0 D`` (all at the
    quantised coefficients), ``dU_n/du_kn = A_k (-i dt H_k) B_k`` exactly because
    H_k commutes with its own exponential.  Hence
    ``d tau/du_kn = -i dt Tr(H_k B_k X_{n-1} U_T^dag L_n A_k)`` and
    ``dF/du_kn = (2/N^2) Re(conj(tau) d tau/du_kn)``.

    Everything is formed explicitly from these definitions (no recursion).
    ``g`` has shape (M, K), units 1/(rad/s).
    """
    M, K, _ = digits_bm.shape
    N = D.shape[0]
    I = np.eye(N, dtype=np.complex128)
    steps = [step_propagator(T, D, digits_bm[n]) for n in range(M)]
    X = [I]                                  # X[n] = U_n ... U_1, X[0] = I
    for n in range(M):
        X.append(steps[n] @ X[-1])
    Lsuf = [None] * (M + 1)                  # Lsuf[n] = U_M ... U_{n+1}
    Lsuf[M] = I
    for n in range(M - 1, -1, -1):
        Lsuf[n] = Lsuf[n + 1] @ steps[n]
    U = X[M]
    tau = trace_overlap(U_target, U)
    F = (abs(tau) ** 2) / float(N * N)
    g = np.zeros((M, K), dtype=np.float64)
    UTd = U_target.conj().T
    for n in range(M):
        E = step_factors(T, D, digits_bm[n])
        # B_k = E_k ... E_0 D ; A_k = E_{K-1} ... E_{k+1}
        Bk = []
        acc = D
        for k in range(K):
            acc = E[k] @ acc
            Bk.append(acc)
        Ak = [None] * K
        acc = I
        for k in range(K - 1, -1, -1):
            Ak[k] = acc
            acc = acc @ E[k]
        Y = X[n] @ UTd @ Lsuf[n + 1]         # X_{n-1} U_T^dag L_n  (0-based step n is step n+1)
        for k in range(K):
            W = Bk[k] @ Y @ Ak[k]
            dtau = -1j * dt * np.trace(Hk[k] @ W)
            g[n, k] = 2.0 / (N * N) * (np.conj(tau) * dtau).real
    return F, g


def state_transfer_gradient(T, D, Hk, dt, digits_bm, psi0, psiT):
    """``(F_S, g)``: the state-transfer fidelity ``F_S = |<psi_T| U |psi0>|^2`` (Section III's
    state-to-state fidelity) and ``g[n][k] = dF_S/du_kn`` of the split model at the quantised
    point, from the same factorisation as :func:`grape_gradient`:
    ``a = <psi_T| U |psi0>``, ``da/du_kn = -i dt <psi_T| L_n A_k H_k B_k X_{n-1} |psi0>``,
    ``dF_S/du_kn = 2 Re(conj(a) da/du_kn)``.  Formed explicitly (no recursion).
    """
    M, K, _ = digits_bm.shape
    N = D.shape[0]
    I = np.eye(N, dtype=np.complex128)
    steps = [step_propagator(T, D, digits_bm[n]) for n in range(M)]
    X = [I]
    for n in range(M):
        X.append(steps[n] @ X[-1])
    Lsuf = [None] * (M + 1)
    Lsuf[M] = I
    for n in range(M - 1, -1, -1):
        Lsuf[n] = Lsuf[n + 1] @ steps[n]
    psi0 = np.asarray(psi0, dtype=np.complex128)
    bra = np.conj(np.asarray(psiT, dtype=np.complex128))
    a = complex(bra @ (X[M] @ psi0))
    F = abs(a) ** 2
    g = np.zeros((M, K), dtype=np.float64)
    for n in range(M):
        E = step_factors(T, D, digits_bm[n])
        Bk = []
        acc = D
        for k in range(K):
            acc = E[k] @ acc
            Bk.append(acc)
        Ak = [None] * K
        acc = I
        for k in range(K - 1, -1, -1):
            Ak[k] = acc
            acc = acc @ E[k]
        for k in range(K):
            da = -1j * dt * complex(bra @ (Lsuf[n + 1] @ Ak[k] @ Hk[k] @ Bk[k] @ X[n] @ psi0))
            g[n, k] = 2.0 * (np.conj(a) * da).real
    return F, g


# ---------------------------------------------------------------------------
# GRAPE update (Section III, flowchart Fig. fc; the paper leaves the rule open)
# ---------------------------------------------------------------------------
# The flowchart evaluates the fidelity and its gradient with REDO propagators,
# changes the controls, and repeats.  It fixes neither the step rule nor how the
# controls are kept inside the coefficient range.  The reading taken here: plain
# ascent along dF/du with a per-pulse step factor (halved when a pulse's
# fidelity fell, grown by 1.1 up to 8 otherwise), or Adam moments per
# coefficient; either way the new coefficient is clipped to the ends [lo_k,
# hi_k] of its level grid, so that it always has a level.

def grape_update(u, g, step, scale, lo, hi):
    """One ascent step ``u_bnk <- clip(u_bnk + step * s_b * g_bnk, lo_k, hi_k)``: the update box
    of the GRAPE flowchart (Section III, Fig. fc), whose rule the paper leaves open.

    ``u``, ``g``: (B, M, K); ``scale``: (B,) per-pulse factors s_b (None: all 1);
    ``lo``, ``hi``: (K,).  Returns the new array (the input is not modified).
    """
    u = np.asarray(u, dtype=np.float64)
    B, M, K = u.shape
    out = np.empty_like(u)
    for b in range(B):
        s_b = 1.0 if scale is None else float(scale[b])
        for k in range(K):
            x = u[b, :, k] + step * s_b * g[b, :, k]
            out[b, :, k] = np.minimum(np.maximum(x, lo[k]), hi[k])
    return out


def grape_step_scale(scale, F, F_prev):
    """Per-pulse step factors of the GRAPE update (Section III, Fig. fc; rule read here):
    ``s_b / 2`` where the
    fidelity fell (``F_b < F_prev_b``), else ``min(1.1 s_b, 8)``; unchanged before
    the first comparison (``F_prev`` None)."""
    scale = np.asarray(scale, dtype=np.float64)
    if F_prev is None:
        return scale.copy()
    out = np.empty_like(scale)
    for b in range(scale.shape[0]):
        out[b] = scale[b] * 0.5 if F[b] < F_prev[b] else min(scale[b] * 1.1, 8.0)
    return out


def grape_adam_update(u, g, m, v, t, lr, lo, hi, beta1=0.9, beta2=0.999, eps=1e-12):
    """One Adam ascent step (Kingma & Ba 2015, ascending instead of descending) on
    every coefficient, step number ``t >= 1``:
    ``m <- b1 m + (1-b1) g``, ``v <- b2 v + (1-b2) g^2``,
    ``u <- clip(u + lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps), lo_k, hi_k)``.
    Returns ``(u, m, v)`` (new arrays)."""
    u = np.asarray(u, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    x = u + lr * m_hat / (np.sqrt(v_hat) + eps)
    K = u.shape[-1]
    out = np.empty_like(u)
    for k in range(K):
        out[..., k] = np.minimum(np.maximum(x[..., k], lo[k]), hi[k])
    return out, m, v


def lbfgs_direction(g, pairs):
    """Ascent direction ``d = H g`` of F by the L-BFGS two-loop recursion (Nocedal & Wright,
    Numerical Optimization, 2nd ed., Algorithm 7.4) for the function f = -F, whose gradient is
    -g.  ``pairs`` lists ``(s_i, y_i)`` oldest first, ``s_i = u_{i+1} - u_i`` and
    ``y_i = -(g_{i+1} - g_i)`` (the change of f's gradient), each with ``s_i . y_i > 0``.  The
    initial matrix is ``gamma I`` with ``gamma = s.y / y.y`` of the newest pair.  With no pairs
    the direction is g itself.  Vectors are flat numpy arrays."""
    q = -np.asarray(g, dtype=np.float64)                  # gradient of f
    if not pairs:
        return -q
    rho = [1.0 / float(np.dot(s, y)) for s, y in pairs]
    alpha = [0.0] * len(pairs)
    for i in range(len(pairs) - 1, -1, -1):
        s, y = pairs[i]
        alpha[i] = rho[i] * float(np.dot(s, q))
        q = q - alpha[i] * y
    s, y = pairs[-1]
    r = (float(np.dot(s, y)) / float(np.dot(y, y))) * q
    for i in range(len(pairs)):
        s, y = pairs[i]
        beta = rho[i] * float(np.dot(y, r))
        r = r + (alpha[i] - beta) * s
    return -r                                              # descent for f = ascent for F


def grape_lbfgs_step(u_trial, g_trial, F_trial, state, lo, hi, history=8, step0=0.05, c1=1e-4,
                     first=False):
    """One step of projected L-BFGS ascent with Armijo backtracking for one pulse (the GRAPE
    update read as a quasi-Newton method; the paper leaves the rule open).

    ``u_trial`` (M, K) is the point just evaluated, with fidelity ``F_trial`` and gradient
    ``g_trial``; ``state`` (a dict, empty on the first call) holds the accepted point ``u``,
    its ``g`` and ``F``, the direction ``d``, the step length ``alpha`` and the pair list.
    Rules, in order:
      * first call: accept the trial point outright;
      * otherwise accept when ``F_trial >= F + c1 * g . (u_trial - u)`` (Armijo, projected step),
        store the pair (s, y) when ``s . y > 0`` (at most ``history``, oldest dropped);
        else halve ``alpha``, and below ``alpha = 1e-3`` drop every pair and restart from the
        gradient;
      * after an accept (or a restart) the direction is :func:`lbfgs_direction`, replaced by the
        gradient (dropping the pairs) when it is not an ascent direction (``g . d <= 0``); a
        gradient direction is scaled so that its largest entry is ``step0`` times the widest
        grid span ``max_k(hi_k - lo_k) / 2``; ``alpha`` restarts at 1;
      * the next trial point is ``clip(u + alpha d, lo_k, hi_k)``.
    Returns ``(u_next, state)``.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ut = np.asarray(u_trial, dtype=np.float64)
    gt = np.asarray(g_trial, dtype=np.float64)
    span = 0.5 * float(np.max(hi - lo))

    def grad_dir(g):
        m = float(np.max(np.abs(g)))
        return g * (step0 * span / m) if m > 0 else np.zeros_like(g)

    new_dir = False
    if first:
        state = {"u": ut.copy(), "g": gt.copy(), "F": float(F_trial), "pairs": []}
        new_dir = True
    else:
        u, g, F = state["u"], state["g"], state["F"]
        p = ut - u
        if float(F_trial) >= F + c1 * float(np.sum(g * p)):
            s = p.ravel()
            y = -(gt - g).ravel()
            if float(np.dot(s, y)) > 0.0:
                state["pairs"] = (state["pairs"] + [(s, y)])[-history:]
            state["u"], state["g"], state["F"] = ut.copy(), gt.copy(), float(F_trial)
            new_dir = True
        else:
            state["alpha"] *= 0.5
            if state["alpha"] < 1e-3:
                state["pairs"] = []
                new_dir = True
    if new_dir:
        g = state["g"]
        if state["pairs"]:
            d = lbfgs_direction(g.ravel(), state["pairs"]).reshape(g.shape)
            if float(np.sum(g * d)) <= 0.0:
                state["pairs"] = []
                d = grad_dir(g)
        else:
            d = grad_dir(g)
        state["d"] = d
        state["alpha"] = 1.0
    x = state["u"] + state["alpha"] * state["d"]
    u_next = np.empty_like(x)
    for k in range(x.shape[-1]):
        u_next[..., k] = np.minimum(np.maximum(x[..., k], lo[k]), hi[k])
    return u_next, state


# ---------------------------------------------------------------------------
# Re-unitarisation
# ---------------------------------------------------------------------------

def polar_unitary(P):
    """Unitary polar factor ``P (P^dag P)^(-1/2)`` via eigen-decomposition of P^dag P: the unitary
    nearest P, which re-unitarisation of finite-precision chains approaches (the paper's chains
    are exact products of unitary operators, Section III; it has no such step)."""
    P = np.asarray(P, dtype=np.complex128)
    w, V = np.linalg.eigh(P.conj().T @ P)
    return P @ ((V * (1.0 / np.sqrt(w))[None, :]) @ V.conj().T)


# ---------------------------------------------------------------------------
# Section IV: expectation values along the chain
# ---------------------------------------------------------------------------

def simulate_expectation(T, D, digits_bm, psi0, obs_diag):
    """``<O>(t_n) = <psi_n| O |psi_n>`` for diagonal O, ``psi_n = U_n ... U_1 psi0``,
    n = 0..M (Section IV, ``Tr[M rho(t)]`` with ``rho = |psi><psi|``).

    Returns ``(expect[M+1], U_final)`` where ``U_final = U_M ... U_1``.
    """
    N = D.shape[0]
    X = np.eye(N, dtype=np.complex128)
    out = np.empty(digits_bm.shape[0] + 1, dtype=np.float64)
    psi = X @ psi0
    out[0] = float(np.sum(obs_diag * (psi.real ** 2 + psi.imag ** 2)))
    for n in range(digits_bm.shape[0]):
        X = step_propagator(T, D, digits_bm[n]) @ X
        psi = X @ psi0
        out[n + 1] = float(np.sum(obs_diag * (psi.real ** 2 + psi.imag ** 2)))
    return out, X


def expect_mixed(T, D, digits_bm, rho0, obs):
    """``Tr[rho(t_n) O]`` with ``rho(t_n) = U_n ... U_1 rho0 (U_n ... U_1)^dag``, n = 0..M, for a
    Hermitian (mixed or deviation) initial density matrix and a Hermitian observable, both
    dense (Section IV, the order parameter of the noisy exotic-freezing study).

    Returns ``(expect[M+1], U_final)``.
    """
    N = D.shape[0]
    X = np.eye(N, dtype=np.complex128)
    out = np.empty(digits_bm.shape[0] + 1, dtype=np.float64)
    out[0] = float(np.trace(rho0 @ obs).real)
    for n in range(digits_bm.shape[0]):
        X = step_propagator(T, D, digits_bm[n]) @ X
        out[n + 1] = float(np.trace(X @ rho0 @ X.conj().T @ obs).real)
    return out, X


# ---------------------------------------------------------------------------
# Learned warm start: FP64 MLP (no counterpart in the paper)
# ---------------------------------------------------------------------------

def gelu(x):
    """Exact GELU ``0.5 x (1 + erf(x / sqrt 2))``, the activation of the warm-start network (an
    extension of the Section III GRAPE application; the paper has no network)."""
    from math import erf
    v = np.vectorize(erf, otypes=[np.float64])
    return 0.5 * x * (1.0 + v(x / math.sqrt(2.0)))


def gelu_grad(x):
    """Derivative of the exact GELU: ``Phi(x) + x phi(x)`` (warm-start network, as :func:`gelu`)."""
    from math import erf
    v = np.vectorize(erf, otypes=[np.float64])
    Phi = 0.5 * (1.0 + v(x / math.sqrt(2.0)))
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return Phi + x * phi


def mlp_init(sizes, rng):
    """Weights ``W_l`` (out, in) ~ U[-1/sqrt(in), 1/sqrt(in)], biases zero (warm-start network,
    as :func:`gelu`)."""
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / math.sqrt(a)
        params.append((rng.uniform(-lim, lim, size=(b, a)), np.zeros(b)))
    return params


def mlp_forward(params, x):
    """Hidden layers ``h = GELU(W h + b)``, output ``tanh(W h + b)``; x is (batch, in) (the
    warm-start network of the GRAPE extension, as :func:`gelu`).

    Returns ``(y, cache)`` with the pre-activations needed by :func:`mlp_backward`.
    """
    h = np.asarray(x, dtype=np.float64)
    cache = [h]
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append(z)
        h = np.tanh(z) if li == len(params) - 1 else gelu(z)
        cache.append(h)
    return h, cache


def mlp_backward(params, cache, y_target):
    """Gradients of the loss ``mean((y - y_target)^2)`` (mean over all entries) by the chain rule
    through :func:`mlp_forward` (warm-start network, as :func:`gelu`)."""
    nl = len(params)
    y = cache[-1]
    dh = 2.0 * (y - y_target) / y.size
    grads = [None] * nl
    for li in range(nl - 1, -1, -1):
        z = cache[2 * li + 1]
        h_in = cache[2 * li]
        if li == nl - 1:
            dz = dh * (1.0 - np.tanh(z) ** 2)
        else:
            dz = dh * gelu_grad(z)
        W, _ = params[li]
        grads[li] = (dz.T @ h_in, dz.sum(axis=0))
        dh = dz @ W
    loss = float(np.mean((y - y_target) ** 2))
    return loss, grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
