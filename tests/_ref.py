"""Test helpers: oracle references for a workload (calls only oracle/ and the input generators)."""
import numpy as np

from oracle import redo_oracle as O


def oracle_table(w, method="pade"):
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits, method=method)
    return T, D


def folded(T, D):
    """Oracle table with the drift folded into term 0, digit 0 (the layout the library stores)."""
    Tf = T.copy()
    for c in range(T.shape[2]):
        Tf[0, 0, c] = T[0, 0, c] @ D
    return Tf


def oracle_levels(w, u=None):
    u = w.u if u is None else u
    q, nn, ns = O.quantize(u, w.lo, w.hi, w.levels)
    return q, O.level_digits(q, w.base, w.digits), nn, ns


def oracle_propagators(w, T, D, digits, pulses):
    return np.stack([O.propagate(T, D, digits[b]) for b in pulses])
