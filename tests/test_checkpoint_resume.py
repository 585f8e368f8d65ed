"""Run checkpoints: a GRAPE run stopped, saved, loaded and resumed equals the uninterrupted run,
and the warm-start network round-trips through its file (CPU only).

The loop's host logic -- iteration counting, step factors, Adam's step number and rate decay,
the L-BFGS state buffer, first-reached iterations, early stop -- is checked with deterministic
stand-ins for the library calls it makes (a smooth fidelity with its exact gradient and simple
update rules that keep their state where the real ones do), installed on the binding module for
each test only.
"""
import types

import numpy as np
import pytest
import torch

from paper_1707_02162_gb300 import grape as G
from paper_1707_02162_gb300 import redo

B, M, K = 3, 6, 2
XSTAR = torch.from_numpy(np.random.default_rng(5).uniform(-0.6, 0.6, size=(B, M, K)))


def _fidelity(q):
    x = q.double() / 1000.0
    d = x - XSTAR
    F = torch.exp(-(d * d).sum(dim=(1, 2)))
    return F, -2.0 * d * F[:, None, None]


def _install(monkeypatch):
    def quantize(h, u, q, status=None, stream=None):
        q.copy_(torch.round(u * 1000.0).to(torch.int32))

    def fidelity_grad(h, q, target, prec, ck, F, g, ws, status=None, reunit_every=0, stream=None):
        Fv, gv = _fidelity(q)
        F.copy_(Fv)
        g.copy_(gv)

    def grape_step(h, u, g, step, scale=None, stream=None):
        s = torch.ones(u.shape[0], dtype=torch.float64) if scale is None else scale
        u.add_(step * s[:, None, None] * g).clamp_(-1.0, 1.0)

    def adam_step(h, u, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-12, stream=None):
        m.mul_(beta1).add_((1 - beta1) * g)
        v.mul_(beta2).add_((1 - beta2) * g * g)
        u.add_(lr * (m / (1 - beta1 ** t)) / (torch.sqrt(v / (1 - beta2 ** t)) + eps)).clamp_(-1.0, 1.0)

    def lbfgs_step(h, u, g, F, state, first, history, step0, c1=1e-4, u_best=None, F_best=None, stream=None):
        # heavy-ball stand-in whose momentum lives in the caller's state buffer
        n = u.numel()
        mom = state[:8 * n].view(torch.float64).view(u.shape)
        if first:
            mom.zero_()
            F_best.fill_(-1.0)
        better = F >= F_best
        u_best[better] = u[better]
        F_best.copy_(torch.where(better, F, F_best))
        mom.mul_(0.5).add_(g)
        u.copy_(u_best + step0 * mom).clamp_(-1.0, 1.0)

    monkeypatch.setattr(redo, "redo_quantize", quantize)
    monkeypatch.setattr(redo, "redo_fidelity_grad", fidelity_grad)
    monkeypatch.setattr(redo, "redo_fidelity_grad_workspace", lambda h, B, M, prec, ck=0: 0)
    monkeypatch.setattr(redo, "redo_grape_step", grape_step)
    monkeypatch.setattr(redo, "redo_grape_adam_step", adam_step)
    monkeypatch.setattr(redo, "redo_grape_lbfgs_workspace", lambda h, B_, M_, hist=8: 8 * B_ * M_ * K + 256)
    monkeypatch.setattr(redo, "redo_grape_lbfgs_step", lbfgs_step)


TABLE = types.SimpleNamespace(handle=0, device=torch.device("cpu"))
TARGET = np.eye(2, dtype=complex)
STEPS = {"gd": 0.05, "adam": 0.02, "lbfgs": 0.1}


def _u0():
    return torch.zeros((B, M, K), dtype=torch.float64)


def _same(a, b):
    assert a.iterations == b.iterations
    assert torch.equal(a.u, b.u) and torch.equal(a.reached, b.reached)
    assert torch.equal(torch.stack(a.F_history), torch.stack(b.F_history))
    for k, v in a.state.items():
        w = b.state[k]
        assert (torch.equal(v, w) if isinstance(v, torch.Tensor) else v == w), k


@pytest.mark.parametrize("opt", ["gd", "adam", "lbfgs"])
def test_resumed_run_equals_the_uninterrupted_run(opt, monkeypatch, tmp_path):
    _install(monkeypatch)
    full = G.grape(TABLE, TARGET, _u0(), iters=12, step=STEPS[opt], optimizer=opt)
    first = G.grape(TABLE, TARGET, _u0(), iters=5, step=STEPS[opt], optimizer=opt)
    assert first.state["iteration"] == 5
    G.save_state(str(tmp_path / "run.npz"), first.state)
    state = G.load_state(str(tmp_path / "run.npz"))
    rest = G.grape(TABLE, TARGET, None, iters=7, step=STEPS[opt], optimizer=opt, resume=state)
    _same(full, rest)
    assert full.F_history[-1].mean() > full.F_history[0].mean()     # the stand-in run does ascend


def test_resume_across_an_early_stop(monkeypatch, tmp_path):
    # the uninterrupted run stops on the threshold; a run cut earlier and resumed stops at the
    # same iteration with the same coefficients and first-reached iterations
    _install(monkeypatch)
    th = 0.6
    full = G.grape(TABLE, TARGET, _u0(), iters=200, step=0.05, threshold=th)
    assert full.iterations < 200 and bool((full.reached >= 0).all())
    cut = full.iterations // 2
    first = G.grape(TABLE, TARGET, _u0(), iters=cut, step=0.05, threshold=th)
    G.save_state(str(tmp_path / "run.npz"), first.state)
    rest = G.grape(TABLE, TARGET, None, iters=200 - cut, step=0.05, threshold=th,
                   resume=G.load_state(str(tmp_path / "run.npz")))
    _same(full, rest)


def test_resume_refuses_another_optimizer(monkeypatch):
    _install(monkeypatch)
    st = G.grape(TABLE, TARGET, _u0(), iters=2, step=0.02, optimizer="adam").state
    with pytest.raises(ValueError, match="resumed with optimizer"):
        G.grape(TABLE, TARGET, None, iters=2, step=0.02, optimizer="gd", resume=st)


def test_mlp_checkpoint_round_trip(tmp_path):
    from paper_1707_02162_gb300.warmstart import MLP
    net = MLP([5, 7, 3], seed=2, device="cpu")
    g = torch.Generator().manual_seed(0)
    net.m.copy_(torch.rand(net.m.shape, generator=g))
    net.v.copy_(torch.rand(net.v.shape, generator=g))
    net.step_count = 17
    net.save(str(tmp_path / "mlp.npz"))
    back = MLP.load(str(tmp_path / "mlp.npz"), device="cpu")
    assert back.sizes == [5, 7, 3] and back.step_count == 17
    for a, b in ((net.params, back.params), (net.m, back.m), (net.v, back.v)):
        assert torch.equal(a, b)
