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


class LazyTable:
    """The oracle's table ``T[k][j][c] = exp(-i dt theta_kjc H_k)`` (eigen-decomposition form), each
    entry evaluated when first indexed: for large N, where the whole table would take hours on the
    CPU and a test touches a few thousand entries."""

    def __init__(self, w):
        self.w = w
        self.th = [O.table_thetas(w.lo[k], w.hi[k], w.levels, w.base, w.digits) for k in range(w.Hk.shape[0])]
        self.eig = [np.linalg.eigh(w.Hk[k]) for k in range(w.Hk.shape[0])]
        self.cache = {}

    def __getitem__(self, idx):
        k, j, c = (int(i) for i in idx)
        if (k, j, c) not in self.cache:
            self.cache[(k, j, c)] = O.expm_hermitian(self.w.Hk[k], self.w.dt * self.th[k][j, c], eig=self.eig[k])
        return self.cache[(k, j, c)]

    def factor(self, k, theta):
        """``exp(-i dt theta H_k)`` for any coefficient theta (finite differences)."""
        return O.expm_hermitian(self.w.Hk[k], self.w.dt * theta, eig=self.eig[k])
