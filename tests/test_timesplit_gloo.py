"""Time-split host logic on CPU ranks (gloo): one pulse cut into time segments, one per rank;
the ordered all-gather, the prefix/suffix regrouping and the per-segment gradient against the
transformed target, with the CPU oracle standing in for the device arithmetic."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import redo_oracle as O


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleOps:
    """Segment products, batched products and local gradients by the CPU oracle."""

    def __init__(self, w):
        self.w = w
        self.T, self.D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)

    def _digits(self, q_local):
        return O.level_digits(q_local.numpy(), self.w.base, self.w.digits)

    def segment_product(self, q_local):
        dig = self._digits(q_local)
        return torch.from_numpy(np.stack([O.propagate(self.T, self.D, dig[b]) for b in range(dig.shape[0])]))

    def product(self, A, B, adjA=False, adjB=False):
        a, b = A.numpy(), B.numpy()
        if adjA:
            a = np.conj(np.swapaxes(a, -1, -2))
        if adjB:
            b = np.conj(np.swapaxes(b, -1, -2))
        return torch.from_numpy(np.ascontiguousarray(a @ b))

    def local_grad(self, q_local, targets):
        dig = self._digits(q_local)
        res = [O.grape_gradient(self.T, self.D, self.w.Hk, self.w.dt, dig[b], targets[b].numpy())
               for b in range(dig.shape[0])]
        return torch.tensor([r[0] for r in res]), torch.from_numpy(np.stack([r[1] for r in res]))


def _workload():
    from paper_1707_02162_gb300 import inputs
    return inputs.config(0, B=2, M=11, base=16, digits=2)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_1707_02162_gb300 import timesplit
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _workload()
    ops = OracleOps(w)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    n0, n1 = timesplit.segment_bounds(w.M, world, rank)
    q_local = torch.from_numpy(np.ascontiguousarray(q[:, n0:n1]))
    U = timesplit.propagate_split(ops, q_local)
    F, g = timesplit.fidelity_grad_split(ops, q_local, torch.from_numpy(w.target))
    out[rank] = (U.numpy(), F.numpy(), g.numpy(), n0, n1)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_time_split_matches_the_whole_pulse(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    w = _workload()
    T, D = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    q, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(q, w.base, w.digits)
    covered = []
    for r in range(world):
        U, F, g, n0, n1 = out[r]
        covered += list(range(n0, n1))
        for b in range(w.B):
            Uo = O.propagate(T, D, dig[b])
            Fo, go = O.grape_gradient(T, D, w.Hk, w.dt, dig[b], w.target)
            assert np.abs(U[b] - Uo).max() < 1e-13
            assert abs(F[b] - Fo) < 1e-13
            assert np.abs(g[b] - go[n0:n1]).max() <= 1e-10 * np.abs(go).max()
    assert covered == list(range(w.M))


def test_segment_bounds_cover_the_pulse():
    from paper_1707_02162_gb300.timesplit import segment_bounds
    for M in (0, 1, 7, 1000):
        for G in (1, 2, 3, 8):
            b = [segment_bounds(M, G, r) for r in range(G)]
            assert b[0][0] == 0 and b[-1][1] == M
            assert all(b[r][1] == b[r + 1][0] for r in range(G - 1))
            assert max(n1 - n0 for n0, n1 in b) - min(n1 - n0 for n0, n1 in b) <= 1
