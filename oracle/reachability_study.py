"""Oracle-side reachability of the learned-warm-start targets -- TEST INFRASTRUCTURE ONLY.

Runs GRAPE on single instances of the warm-start system (5 qubits, N=32, K=10 per-qubit x/y
controls, M=500 steps of 2 us, 4096 levels, every instance its own offsets nu ~ U[-5, 5] kHz and
couplings J ~ U[-200, 200] Hz) entirely in the FP64 oracle, to tell what the problem allows from
what an optimiser reaches:

* ``--optimizer lbfgsb``: scipy's L-BFGS-B on 1 - F, F and dF/du from the oracle at the quantised
  coefficients (the straight-through gradient of the GPU path), bounds = the level grid, with its
  gradient and relative-reduction stopping tests made negligible (a start far from the target has
  a tiny gradient);
* ``--optimizer adam``: the oracle's own Adam ascent (``grape_adam_update``) with a learning rate
  lr * Omega / (1 + it / decay).

Targets exp(-i sum_k theta_k P_k), theta ~ U[0, theta_max], over 8 Pauli strings drawn once from
seed 4: weight-one strings (``--family local``) or uniformly random non-identity strings
(``--family random``).  Usage::

    python -m oracle.reachability_study --family local --instance 0 --optimizer lbfgsb --evals 600

Prints the fidelity every 50 evaluations and the first evaluation at F >= 0.999.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import redo_oracle as O  # noqa: E402
from paper_1707_02162_gb300 import inputs  # noqa: E402  (seeded input generators only)


def _strings(family, n, rng):
    out = []
    while len(out) < 8:
        if family == "local":
            s = ["I"] * n
            s[int(rng.integers(n))] = "XYZ"[int(rng.integers(3))]
            s = "".join(s)
        else:
            s = "".join("IXYZ"[int(c)] for c in rng.integers(0, 4, size=n))
        if s != "I" * n and s not in out:
            out.append(s)
    return out


def instance(family: str, idx: int, theta_max: float):
    """(w, T, D, U_target, u0) of one instance (oracle table with that instance's drift)."""
    w = inputs.config(4, B=1)
    n = w.n_qubits
    strings = _strings(family, n, np.random.default_rng(4))
    rng = np.random.default_rng(100 + idx)
    theta = rng.uniform(0.0, theta_max, size=8)
    G = inputs.pauli_generator(strings, theta)
    UT = O.expm_pade13(-1j * G)
    iu = np.triu_indices(n, 1)
    nu = rng.uniform(-5e3, 5e3, size=n)
    Jm = np.zeros((n, n))
    Jm[iu] = rng.uniform(-200.0, 200.0, size=iu[0].size)
    H0 = inputs.drift_zz(n, nu, Jm)
    T, D = O.build_table(H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits, method="eig")
    Om = w.extra["Omega"]
    u0 = rng.uniform(-0.3 * Om, 0.3 * Om, size=(w.M, w.K))
    return w, T, D, UT, u0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--family", choices=["local", "random"], default="local")
    ap.add_argument("--instance", type=int, default=0)
    ap.add_argument("--theta-max", type=float, default=np.pi)
    ap.add_argument("--optimizer", choices=["lbfgsb", "adam"], default="lbfgsb")
    ap.add_argument("--evals", type=int, default=600)
    ap.add_argument("--lr", type=float, default=0.01, help="adam: learning rate in units of Omega")
    ap.add_argument("--decay", type=float, default=150.0, help="adam: rate decays as 1 / (1 + it / decay)")
    a = ap.parse_args(argv)
    w, T, D, UT, u0 = instance(a.family, a.instance, a.theta_max)
    Om = w.extra["Omega"]
    t0, count, first = time.time(), [0], [-1]

    def fg(u):
        q, _, _ = O.quantize(u[None], w.lo, w.hi, w.levels)
        F, g = O.grape_gradient(T, D, w.Hk, w.dt, O.level_digits(q, w.base, w.digits)[0], UT)
        count[0] += 1
        if F >= 0.999 and first[0] < 0:
            first[0] = count[0]
        if count[0] % 50 == 0:
            print(f"{a.family} {a.instance} {a.optimizer} eval {count[0]} F {F:.6f} ({time.time() - t0:.0f} s)",
                  flush=True)
        return F, g

    if a.optimizer == "lbfgsb":
        from scipy.optimize import minimize

        def f_and_grad(x):
            F, g = fg((x * Om).reshape(w.M, w.K))
            return 1.0 - F, -(g * Om).ravel()

        r = minimize(f_and_grad, (u0 / Om).ravel(), jac=True, method="L-BFGS-B",
                     bounds=[(-1.0, 1.0)] * (w.M * w.K),
                     options={"maxiter": a.evals, "maxfun": a.evals, "gtol": 1e-14, "ftol": 1e-15})
        Fend = 1.0 - r.fun
    else:
        u, m, v = u0[None].copy(), np.zeros((1, w.M, w.K)), np.zeros((1, w.M, w.K))
        Fend = 0.0
        for it in range(a.evals):
            Fend, g = fg(u[0])
            u, m, v = O.grape_adam_update(u, g[None], m, v, it + 1, a.lr * Om / (1 + it / a.decay), w.lo, w.hi)
    print(f"done {a.family} {a.instance} {a.optimizer}: {count[0]} evaluations, final F {Fend:.6f}, "
          f"first F >= 0.999 at evaluation {first[0]}", flush=True)


if __name__ == "__main__":
    main()
