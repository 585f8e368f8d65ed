"""Learned warm start for REDO-GRAPE.

A multilayer perceptron maps the parameters of a control problem (target
generator angles and system constants) to an initial pulse in normalised
amplitude (u / Omega in [-1, 1]).  It is trained, with libredo's own forward,
backward and Adam kernels, on pulses that the GPU REDO-GRAPE itself converged,
and judged against plain random-initialised GRAPE by the number of iterations
to reach a fidelity threshold.  The paper has no counterpart; this is the
learned extension of its GRAPE application (Section III).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import redo
from .grape import grape


class MLP:
    """FP32 multilayer perceptron whose arithmetic runs in libredo kernels."""

    def __init__(self, sizes, params: np.ndarray | None = None, seed: int = 0, device="cuda"):
        self.sizes = [int(s) for s in sizes]
        self.device = torch.device(device)
        n, _, _ = redo.redo_mlp_sizes(self.sizes, 1)
        if params is None:
            rng = np.random.default_rng(seed)
            chunks = []
            for a, b in zip(self.sizes[:-1], self.sizes[1:]):
                lim = 1.0 / np.sqrt(a)
                chunks += [rng.uniform(-lim, lim, size=b * a), np.zeros(b)]
            params = np.concatenate(chunks)
        assert params.size == n
        self.params = torch.tensor(params, dtype=torch.float32, device=self.device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        self._buf = {}

    def save(self, path: str) -> None:
        """Weights, Adam moments and step count to an ``.npz`` file (training resumes from it)."""
        np.savez(path, sizes=np.array(self.sizes, dtype=np.int64), params=self.params.cpu().numpy(),
                 m=self.m.cpu().numpy(), v=self.v.cpu().numpy(), step_count=np.array(self.step_count))

    @classmethod
    def load(cls, path: str, device="cuda") -> "MLP":
        """The network saved by :meth:`save`, ready to continue training where it stopped."""
        with np.load(path) as z:
            net = cls([int(s) for s in z["sizes"]], params=z["params"].astype(np.float64), device=device)
            net.m.copy_(torch.from_numpy(z["m"]))
            net.v.copy_(torch.from_numpy(z["v"]))
            net.step_count = int(z["step_count"])
        return net

    def _buffers(self, batch):
        if batch not in self._buf:
            _, na, nw = redo.redo_mlp_sizes(self.sizes, batch)
            self._buf[batch] = (torch.empty(max(na, 1), dtype=torch.float32, device=self.device),
                                torch.empty(max(nw, 1), dtype=torch.float32, device=self.device),
                                torch.empty((batch, self.sizes[-1]), dtype=torch.float32, device=self.device))
        return self._buf[batch]

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.to(self.device, torch.float32).contiguous()
        acts, _, y = self._buffers(x.shape[0])
        redo.redo_mlp_forward(self.sizes, self.params, x, acts, y)
        return y.clone()

    def train_step(self, x: torch.Tensor, y_target: torch.Tensor, lr: float) -> float:
        x = x.to(self.device, torch.float32).contiguous()
        y_target = y_target.to(self.device, torch.float32).contiguous()
        acts, work, y = self._buffers(x.shape[0])
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        redo.redo_mlp_forward(self.sizes, self.params, x, acts, y)
        redo.redo_mlp_backward(self.sizes, self.params, x, acts, y_target, self.grads, loss, work)
        self.step_count += 1
        redo.redo_mlp_adam(self.params, self.grads, self.m, self.v, self.step_count, lr)
        return float(loss.item())


@dataclass
class WarmStartReport:
    train_instances: int
    test_instances: int
    threshold: float
    random_iters: list
    mlp_iters: list
    final_loss: float
    random_F0: float = float("nan")     # median fidelity of the initial pulses
    mlp_F0: float = float("nan")
    random_Fend: float = float("nan")   # median fidelity after the iteration budget
    mlp_Fend: float = float("nan")

    def summary(self) -> dict:
        def med(v, q=50):
            a = np.array([x if x >= 0 else np.inf for x in v], dtype=float)
            # an element of the list (instances that never reached the threshold count as infinite)
            return float(np.percentile(a, q, method="higher")) if a.size else float("nan")

        def med_reached(v):
            a = np.array([x for x in v if x >= 0], dtype=float)
            return float(np.median(a)) if a.size else float("nan")
        return {"threshold": self.threshold, "train": self.train_instances, "test": self.test_instances,
                "median_iters_random_init": med(self.random_iters), "median_iters_mlp_init": med(self.mlp_iters),
                "p25_iters_random_init": med(self.random_iters, 25), "p25_iters_mlp_init": med(self.mlp_iters, 25),
                "median_iters_among_reached_random": med_reached(self.random_iters),
                "median_iters_among_reached_mlp": med_reached(self.mlp_iters),
                "reached_random": int(sum(x >= 0 for x in self.random_iters)),
                "reached_mlp": int(sum(x >= 0 for x in self.mlp_iters)), "final_train_loss": self.final_loss,
                "median_F_initial_random": self.random_F0, "median_F_initial_mlp": self.mlp_F0,
                "median_F_final_random": self.random_Fend, "median_F_final_mlp": self.mlp_Fend}


def converge(table: redo.Table, targets: np.ndarray, u0: np.ndarray, iters: int, step: float, threshold: float,
             prec="fp64", optimizer="gd", drift=None, chunk: int = 256, reunit_every: int = 0):
    """Batched GRAPE on per-instance targets (and, with ``drift`` [B][N], per-instance diagonal
    drifts), ``chunk`` instances per batch (so that every forward state of a batch stays kept);
    returns (u, first iteration reaching threshold per instance, fidelity history [iters][B])."""
    us, reached, hist = [], [], []
    for a in range(0, len(u0), chunk):
        b = min(a + chunk, len(u0))
        res = grape(table, torch.as_tensor(targets[a:b], device=table.device),
                    torch.as_tensor(u0[a:b], device=table.device), iters=iters, step=step, prec=prec,
                    threshold=threshold, optimizer=optimizer, drift=None if drift is None else drift[a:b],
                    checkpoint_every=reunit_every, reunit_every=reunit_every)
        us.append(res.u)
        reached += res.reached.tolist()
        F = torch.stack(res.F_history)
        if F.shape[0] < iters:                 # stopped early: every instance reached; hold the last values
            F = torch.cat([F, F[-1:].expand(iters - F.shape[0], -1)])
        hist.append(F)
    return torch.cat(us), reached, torch.cat(hist, dim=1)


def local_pauli_family(n_qubits: int, n_strings: int, rng: np.random.Generator) -> list[str]:
    """Weight-one Pauli strings (one X, Y or Z on one qubit): targets built from them are
    products of single-qubit rotations, reachable with per-qubit x/y controls."""
    out = []
    while len(out) < n_strings:
        qb = int(rng.integers(n_qubits))
        s = ["I"] * n_qubits
        s[qb] = "XYZ"[int(rng.integers(3))]
        s = "".join(s)
        if s not in out:
            out.append(s)
    return out


def study(table: redo.Table, n_qubits: int, M: int, K: int, Omega: float, features_const: np.ndarray | None = None,
          n_train: int = 512, n_test: int = 64, threshold: float = 0.99, iters: int = 400, step: float = 0.0,
          theta_max: float = np.pi, train_steps: int = 1500, hidden=(512, 512, 512), seed: int = 4,
          prec: str = "fp32", per_instance_drift: bool = False, optimizer: str = "lbfgs",
          reunit_every: int = 50, train_threshold: float | None = None) -> WarmStartReport:
    """Learned warm start: targets exp(-i sum_k theta_k P_k) over a fixed set of Pauli strings;
    MLP input = (system constants, theta); output = M*K normalised amplitudes.

    ``per_instance_drift=False``: one system, the table's own drift, whose constants
    ``features_const`` head every input.  ``per_instance_drift=True``: the table must be built
    with H0 = 0; every instance draws its own offsets nu ~ U[-5, 5] kHz and couplings
    J ~ U[-200, 200] Hz (i < j), GRAPE runs with that diagonal drift per instance, and the input
    is (nu / 5 kHz, J / 200 Hz, theta): for 5 qubits 5 + 10 + 8 = 23 numbers.

    ``optimizer``: "lbfgs" (``step`` = size of a gradient step as a fraction of half the grid,
    default 0.05) or "adam" (``step`` = learning rate in rad/s, default 0.01 Omega).  Reduced
    precision chains are re-unitarised every ``reunit_every`` steps (their checkpoint segments).
    The training pulses are converged to ``train_threshold`` (default: ``threshold``) and the
    ones that reach it are the training set; the test instances run the whole budget from both
    starts and report the first iteration at ``threshold``."""
    from scipy.linalg import expm as _expm   # target construction only (problem input)
    from .inputs import drift_zz, pauli_generator
    rng = np.random.default_rng(seed)
    strings = local_pauli_family(n_qubits, 8, rng)
    lr = step if step > 0 else (0.05 if optimizer == "lbfgs" else 0.01 * Omega)
    ru = reunit_every if prec != "fp64" else 0
    iu = np.triu_indices(n_qubits, 1)

    def targets(count):
        th = rng.uniform(0.0, theta_max, size=(count, len(strings)))
        T = np.stack([_expm(-1j * pauli_generator(strings, t)) for t in th])
        return th, T

    def systems(count):
        """(system features [count][F], diagonal drifts [count][N] or None)."""
        if not per_instance_drift:
            return np.broadcast_to(features_const, (count, features_const.size)), None
        nu = rng.uniform(-5e3, 5e3, size=(count, n_qubits))
        J = rng.uniform(-200.0, 200.0, size=(count, iu[0].size))
        h = np.empty((count, 2 ** n_qubits))
        for b in range(count):
            Jm = np.zeros((n_qubits, n_qubits))
            Jm[iu] = J[b]
            h[b] = np.real(np.diag(drift_zz(n_qubits, nu[b], Jm)))
        return np.concatenate([nu / 5e3, J / 200.0], axis=1), h

    def feats(sysf, th):
        return torch.tensor(np.concatenate([sysf, th / theta_max * 2 - 1], axis=1), dtype=torch.float32)

    th_tr, T_tr = targets(n_train)
    sys_tr, h_tr = systems(n_train)
    # every training instance starts from the same pulse, so that the converged pulses
    # follow one smooth branch of solutions in theta (what the network can learn)
    u0 = np.broadcast_to(rng.uniform(-0.3 * Omega, 0.3 * Omega, size=(1, M, K)), (n_train, M, K)).copy()
    thr_tr = threshold if train_threshold is None else train_threshold
    u_tr, reached, _ = converge(table, T_tr, u0, iters, lr, thr_tr, prec, optimizer, drift=h_tr, reunit_every=ru)
    ok = np.array(reached) >= 0
    if not ok.any():
        raise RuntimeError("no training instance reached the threshold; raise iters or lr")
    x = feats(sys_tr[ok], th_tr[ok])
    y = torch.tensor(u_tr.cpu().numpy()[ok].reshape(int(ok.sum()), -1) / Omega, dtype=torch.float32)
    net = MLP([x.shape[1], *hidden, M * K], seed=seed)
    loss = float("nan")
    for _ in range(train_steps):
        loss = net.train_step(x, y, 1e-3)
    th_te, T_te = targets(n_test)
    sys_te, h_te = systems(n_test)
    u_mlp = net.forward(feats(sys_te, th_te)).cpu().numpy().reshape(n_test, M, K).astype(np.float64) * Omega
    u_rnd = rng.uniform(-0.3 * Omega, 0.3 * Omega, size=(n_test, M, K))
    # threshold=None keeps every run to the full budget so the final fidelities compare
    _, _, F_mlp = converge(table, T_te, u_mlp, iters, lr, None, prec, optimizer, drift=h_te, reunit_every=ru)
    _, _, F_rnd = converge(table, T_te, u_rnd, iters, lr, None, prec, optimizer, drift=h_te, reunit_every=ru)

    def first_reach(F):
        hit = F >= threshold                                # F: [iters][B]
        out = []
        for b in range(F.shape[1]):
            idx = torch.nonzero(hit[:, b])
            out.append(int(idx[0]) if idx.numel() else -1)
        return out, float(F[0].median()), float(F[-1].median())
    it_mlp, f0m, fem = first_reach(F_mlp)
    it_rnd, f0r, fer = first_reach(F_rnd)
    return WarmStartReport(int(ok.sum()), n_test, threshold, it_rnd, it_mlp, loss, f0r, f0m, fer, fem)
