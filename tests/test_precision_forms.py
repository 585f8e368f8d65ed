"""Why the product chains offer no plain TF32 form (CPU, no GPU needed).

A TF32 operand keeps 10 explicit significand bits (unit roundoff 2^-11).  Emulated here on the
benchmark's system (N=64, K=12, 4096 levels, b=64, d=2) for 100 steps: every operand of every
complex product is rounded to TF32 and the products accumulate in FP32, as a kind::tf32 tensor-core
chain would, and the product is re-unitarised as the reduced forms are.  Against the FP64 oracle
chain the result is off by ~7e-3 per entry (the split-FP16 and FP32 forms meet 2e-4), and its
fidelity against the benchmark's Haar target moves by ~2e-6 already after these 100 of the 2000
steps (3e-5 against the reached target); the same chain with FP32 operands stays at ~1e-6 and
~1e-10.  A three-product split TF32 form would carry 11 + 11 bits like the split-FP16 form at half
the dense tensor rate and twice the operand bytes, so split FP16 is the reduced form offered.
"""
import numpy as np

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs


def _tf32(x):
    """Round float32 values to TF32 (10 explicit significand bits), nearest with ties to even."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0xFFF + ((a >> 13) & 1)) & ~np.uint64(0x1FFF)
    return a.astype(np.uint32).view(np.float32)


def _ctf32(Z):
    return (_tf32(Z.real) + 1j * _tf32(Z.imag)).astype(np.complex64)


def test_tf32_rounding_helper():
    # 1 + 2^-11 is a tie between 1 and 1 + 2^-10: rounds to even (1); 1 + 3*2^-11 rounds up
    x = np.array([1.0, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 1 + 2.0 ** -10, -1.5], dtype=np.float32)
    assert _tf32(x).tolist() == [1.0, 1.0, 1 + 2.0 ** -9, 1 + 2.0 ** -10, -1.5]


def test_tf32_chain_misses_the_error_budget_fp32_meets_it():
    w = inputs.config(1, B=1, M=100)
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits, method="eig")
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)[0]
    U64 = O.propagate(T, D, dig)
    X32 = np.eye(w.N, dtype=np.complex64)
    Xtf = np.eye(w.N, dtype=np.complex64)
    for n in range(w.M):
        ops = [T[k, j, dig[n, k, j]] for k in range(w.K) for j in range(w.digits)]
        ops[0] = ops[0] @ D                                  # the drift folded into the first factor
        for A in ops:
            X32 = A.astype(np.complex64) @ X32
            Xtf = _ctf32(A) @ _ctf32(Xtf)
    # both products re-unitarised (polar factor), as the reduced-precision chains are, which
    # removes the coherent norm drift of FP32 accumulation and leaves the rounding
    P32 = O.polar_unitary(X32.astype(np.complex128))
    Ptf = O.polar_unitary(Xtf.astype(np.complex128))
    F64 = O.fidelity(w.target, U64)
    assert np.abs(P32 - U64).max() < 1e-5
    assert abs(O.fidelity(U64, P32) - 1.0) < 1e-9
    assert abs(O.fidelity(w.target, P32) - F64) < 1e-8
    assert np.abs(Ptf - U64).max() > 2e-3
    assert abs(O.fidelity(U64, Ptf) - 1.0) > 1e-5
    assert abs(O.fidelity(w.target, Ptf) - F64) > 1e-6       # already at 1/20 of the benchmark's steps
