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

    def summary(self) -> dict:
        def med(v):
            a = np.array([x if x >= 0 else np.inf for x in v], dtype=float)
            return float(np.median(a))
        return {"threshold": self.threshold, "train": self.train_instances, "test": self.test_instances,
                "median_iters_random_init": med(self.random_iters), "median_iters_mlp_init": med(self.mlp_iters),
                "reached_random": int(sum(x >= 0 for x in self.random_iters)),
                "reached_mlp": int(sum(x >= 0 for x in self.mlp_iters)), "final_train_loss": self.final_loss}


def converge(table: redo.Table, targets: np.ndarray, u0: np.ndarray, iters: int, step: float, threshold: float,
             prec="fp64"):
    """Batched GRAPE on per-instance targets; returns (u, first iteration reaching threshold per instance)."""
    res = grape(table, torch.as_tensor(targets, device=table.device), torch.as_tensor(u0, device=table.device),
                iters=iters, step=step, prec=prec, threshold=threshold)
    return res.u, res.reached.tolist(), res
