"""One long pulse cut into time segments across ranks (a single exchange step).

Rank r of G owns the contiguous steps ``[n0, n1)`` of every pulse and forms its segment product
``S_r = U_{n1} ... U_{n0+1}`` on its own GPU.  One ordered all-gather of the G segment products
gives every rank the whole propagator ``U = S_{G-1} ... S_0`` (Section III's chain regrouped; only
rounding changes).  For the GRAPE gradient, rank r forms its prefix ``P_r = S_{r-1} ... S_0`` and
suffix ``L_r = S_{G-1} ... S_{r+1}`` from the gathered products and differentiates its own
segment against the target ``L_r^dag U_T P_r^dag``: the unitary fidelity is unchanged by that
regrouping, ``Tr(U_T^dag L S P) = Tr((L^dag U_T P^dag)^dag S)``, so the local gradient of the
segment's controls is the full gradient's slice.

The arithmetic goes through an ``ops`` object: :class:`LibraryOps` (libredo on the device) is the
product path; tests may pass another implementation with the same three methods.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def segment_bounds(M: int, world: int, rank: int) -> tuple[int, int]:
    """Steps ``[n0, n1)`` of rank ``rank``: contiguous, sizes differing by at most one."""
    base, extra = divmod(M, world)
    n0 = rank * base + min(rank, extra)
    return n0, n0 + base + (1 if rank < extra else 0)


class LibraryOps:
    """Segment products, batched products and local gradients by libredo (device tensors)."""

    def __init__(self, table, prec: str = "fp64", reunit_every: int = 0, checkpoint_every: int = 0):
        self.table, self.prec = table, prec
        self.reunit_every, self.checkpoint_every = reunit_every, checkpoint_every

    def segment_product(self, q_local: torch.Tensor) -> torch.Tensor:
        U, _, _ = self.table.propagate(q_local, self.prec, reunit_every=self.reunit_every)
        return U

    def product(self, A: torch.Tensor, B: torch.Tensor, adjA: bool = False, adjB: bool = False) -> torch.Tensor:
        from . import redo
        return redo.redo_batched_product(A, B, adjA, adjB)

    def local_grad(self, q_local: torch.Tensor, targets: torch.Tensor):
        return self.table.fidelity_grad(q_local, targets, self.prec, checkpoint_every=self.checkpoint_every)


def combine(ops, segments: list) -> torch.Tensor:
    """``U = S_{G-1} ... S_0`` from the ordered segment products (each [B][N][N])."""
    U = segments[0]
    for S in segments[1:]:
        U = ops.product(S, U)
    return U


def local_target(ops, segments: list, rank: int, target: torch.Tensor) -> torch.Tensor:
    """``L_r^dag U_T P_r^dag`` for every pulse ([B][N][N]); ``target`` is [N][N] or [B][N][N]."""
    G = len(segments)
    B = segments[0].shape[0]
    T = target if target.dim() == 3 else target.unsqueeze(0).expand(B, -1, -1)
    if rank < G - 1:
        L = segments[G - 1]
        for i in range(G - 2, rank, -1):
            L = ops.product(L, segments[i])            # S_{G-1} ... S_{i}
        T = ops.product(L, T, adjA=True)
    if rank > 0:
        P = segments[0]
        for i in range(1, rank):
            P = ops.product(segments[i], P)            # S_{i} ... S_0
        T = ops.product(T, P, adjB=True)
    return T


def _all_gather(S: torch.Tensor, group=None) -> list:
    """Ordered all-gather of a complex tensor (exchanged as its real view)."""
    world = dist.get_world_size(group)
    real = torch.view_as_real(S.contiguous())
    bufs = [torch.empty_like(real) for _ in range(world)]
    dist.all_gather(bufs, real, group=group)
    return [torch.view_as_complex(b) for b in bufs]


def propagate_split(ops, q_local: torch.Tensor, group=None) -> torch.Tensor:
    """Whole propagators [B][N][N] on every rank from this rank's slice of level indices."""
    return combine(ops, _all_gather(ops.segment_product(q_local), group))


def fidelity_grad_split(ops, q_local: torch.Tensor, target: torch.Tensor, group=None):
    """``(F [B], g_local [B][n1-n0][K])``: the fidelity of the whole pulse and the gradient of
    this rank's steps."""
    segments = _all_gather(ops.segment_product(q_local), group)
    rank = dist.get_rank(group)
    return ops.local_grad(q_local, local_target(ops, segments, rank, target))
