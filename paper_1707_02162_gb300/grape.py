"""GRAPE with REDO propagators on the GPU (Section III, Fig. fc).

* :class:`RedoFidelity` -- ``torch.autograd.Function``: the fidelity of every
  pulse against a target, differentiable with respect to the control
  coefficients through libredo's gradient entry point (the derivative of the
  split model at the quantised point; the quantizer is passed straight through).
* :class:`RedoStateFidelity` -- the same for the state fidelity ``|<psi_T|U|psi0>|^2``.
* :class:`RedoPhaseFidelity` -- the unitary fidelity of amplitude/phase controls (Section III's
  {Omega_kn, phi_kn}), differentiable in both amplitudes and phases.
* :func:`grape` -- the ascent loop: quantise, fidelity + gradient, update in
  place; the table is built once outside the loop as the method prescribes.
  Every step of an iteration runs in libredo kernels; the only host read per
  iteration is the fidelity vector.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import redo


class RedoStateFidelity(torch.autograd.Function):
    """F_S = |<psi_T| U(u) |psi0>|^2 for u of shape [B][M][K], differentiable through libredo's
    state-transfer gradient (matrix-vector sweeps; the quantizer is passed straight through)."""

    @staticmethod
    def forward(ctx, u, table: redo.Table, psi0, psi_target, prec="fp64"):
        q = table.quantize(u.detach())
        F, g = table.state_grad(q, psi0, psi_target, prec)
        ctx.save_for_backward(g)
        return F

    @staticmethod
    def backward(ctx, grad_F):
        (g,) = ctx.saved_tensors
        return grad_F[:, None, None] * g, None, None, None, None


class RedoPhaseFidelity(torch.autograd.Function):
    """F = |Tr(U_T^dag U(A, phi))|^2 / N^2 for amplitudes A and phases phi of shape [B][M][K]
    (one x-table per species, the table's phase axes set); gradients in both through libredo's
    amplitude/phase gradient (the amplitude quantizer is passed straight through)."""

    @staticmethod
    def forward(ctx, amp, phi, table: redo.Table, target, prec="fp64", checkpoint_every=0):
        q = table.quantize(amp.detach())
        F, gA, gP = table.fidelity_grad_phase(q, phi.detach(), target, prec, checkpoint_every)
        ctx.save_for_backward(gA, gP)
        return F

    @staticmethod
    def backward(ctx, grad_F):
        gA, gP = ctx.saved_tensors
        w = grad_F[:, None, None]
        return w * gA, w * gP, None, None, None, None


class RedoFidelity(torch.autograd.Function):
    """F = |Tr(U_T^dag U(u))|^2 / N^2 for u of shape [B][M][K] (float64, device)."""

    @staticmethod
    def forward(ctx, u, table: redo.Table, target, prec="fp64", checkpoint_every=0):
        q = table.quantize(u.detach())
        F, g = table.fidelity_grad(q, target, prec, checkpoint_every)
        ctx.save_for_backward(g)
        return F

    @staticmethod
    def backward(ctx, grad_F):
        (g,) = ctx.saved_tensors
        return grad_F[:, None, None] * g, None, None, None, None


@dataclass
class GrapeResult:
    u: torch.Tensor
    F_history: list = field(default_factory=list)
    iterations: int = 0
    reached: torch.Tensor | None = None        # per pulse: first iteration with F >= threshold (-1 if never)
    state: dict | None = None                  # everything a later grape(..., resume=state) continues from


_STATE_TENSORS = ("u", "scale", "prev_F", "reached", "F_history", "m", "v", "lbfgs_state", "u_best", "F_best")


def save_state(path: str, state: dict) -> None:
    """Write a GRAPE run's state (``GrapeResult.state``) to an ``.npz`` file."""
    import numpy as np
    arrays = {"optimizer": np.array(state["optimizer"]), "iteration": np.array(state["iteration"])}
    for k in _STATE_TENSORS:
        if state.get(k) is not None:
            arrays[k] = state[k].detach().cpu().numpy()
    np.savez(path, **arrays)


def load_state(path: str) -> dict:
    """Read a state written by :func:`save_state` (host tensors; ``grape`` moves them)."""
    import numpy as np
    with np.load(path) as z:
        state = {"optimizer": str(z["optimizer"]), "iteration": int(z["iteration"])}
        for k in _STATE_TENSORS:
            state[k] = torch.from_numpy(z[k].copy()) if k in z.files else None
    return state


def grape(table: redo.Table, target, u0: torch.Tensor, iters: int, step: float, prec="fp64",
          checkpoint_every=0, threshold: float | None = None, adaptive: bool = True,
          optimizer: str = "gd", lr_decay: float = 150.0, psi0=None, drift=None,
          on_iter=None, reunit_every: int = 0, resume: dict | None = None) -> GrapeResult:
    """Gradient ascent on the fidelity (the paper does not specify the update rule).

    ``optimizer="gd"``: ``u <- clamp(u + step * dF/du)``; with ``adaptive`` the
    step of a pulse is halved whenever its fidelity decreased and grown by 1.1
    otherwise.  ``optimizer="adam"``: Adam moments per coefficient, ``step`` is
    then the learning rate in rad/s, decayed as step / (1 + it / lr_decay).
    ``optimizer="lbfgs"``: projected L-BFGS with Armijo backtracking (redo_grape_lbfgs_step,
    8 pairs), ``step`` the size of a gradient step as a fraction of half the widest grid; every
    iteration is one fidelity and gradient evaluation, and the result is the accepted point.
    Stops early once every pulse reached ``threshold``.  With ``psi0`` given, ``target`` is a
    state ([N] or [B][N]) and the objective is the state fidelity |<target| U |psi0>|^2
    (redo_state_grad: matrix-vector sweeps instead of propagators).  With ``drift`` ([B][N], rad/s)
    every pulse carries its own diagonal drift (redo_fidelity_grad_drift; the table's own drift,
    usually zero then, is applied as well).  ``on_iter(it, u, F)``, if given, is called after each
    update with the iteration index, the updated coefficients (device, not copied) and that
    iteration's fidelities (host).  ``reunit_every`` (unitary fidelities; equal to ``checkpoint_every``)
    re-unitarises every checkpoint segment of the reduced-precision chains.

    The result's ``state`` holds the run's position: coefficients, iteration count, fidelity
    history, first-reached iterations and the optimizer's own state (step factors, Adam moments,
    or the L-BFGS pair ring and best point).  ``grape(..., resume=state)`` (``u0`` may then be
    None) continues that run for ``iters`` more iterations with the same ``optimizer``, ``step``
    and ``lr_decay``, exactly as an uninterrupted run would; :func:`save_state` and
    :func:`load_state` keep it in an ``.npz`` file between processes.
    """
    if resume is not None and resume["optimizer"] != optimizer:
        raise ValueError(f"state of a {resume['optimizer']!r} run resumed with optimizer {optimizer!r}")
    dev = u0.device if u0 is not None else table.device
    u = (resume["u"].to(dev) if resume is not None else u0).clone().contiguous()
    B, M, K = u.shape
    scale_h = torch.ones(B, dtype=torch.float64)               # per-pulse step factors (host)
    scale_d = torch.ones(B, dtype=torch.float64, device=u.device)
    prev_F = None
    reached = torch.full((B,), -1, dtype=torch.int64)
    res = GrapeResult(u=u)
    it0 = 0
    if resume is not None:
        it0 = res.iterations = resume["iteration"]
        reached = resume["reached"].clone()
        res.F_history = [f.clone() for f in resume["F_history"]]
        if resume.get("scale") is not None:
            scale_h = resume["scale"].clone()
            scale_d.copy_(scale_h)
        prev_F = resume["prev_F"].clone() if resume.get("prev_F") is not None else None
    state = psi0 is not None
    if state and drift is not None:
        raise ValueError("per-pulse drift is supported for the unitary fidelity only")
    if state:
        nbytes = redo.redo_state_grad_workspace(table.handle, B)
        psi0 = torch.as_tensor(psi0, dtype=torch.complex128, device=u.device).contiguous()
    elif drift is not None:
        drift = torch.as_tensor(drift, dtype=torch.float64, device=u.device).contiguous()
        nbytes = redo.redo_fidelity_grad_drift_workspace(table.handle, B, M, prec, checkpoint_every)
    else:
        nbytes = redo.redo_fidelity_grad_workspace(table.handle, B, M, prec, checkpoint_every)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=u.device)
    target = torch.as_tensor(target, dtype=torch.complex128, device=u.device).contiguous()
    q = torch.empty(u.shape, dtype=torch.int32, device=u.device)
    F = torch.empty(B, dtype=torch.float64, device=u.device)
    g = torch.empty(u.shape, dtype=torch.float64, device=u.device)
    if optimizer == "adam":
        m_ = torch.zeros_like(u)
        v_ = torch.zeros_like(u)
        if resume is not None:
            m_.copy_(resume["m"])
            v_.copy_(resume["v"])
    elif optimizer == "lbfgs":
        lb_state = torch.empty(max(redo.redo_grape_lbfgs_workspace(table.handle, B, M, 8), 256),
                               dtype=torch.uint8, device=u.device)
        u_best = u.clone()
        F_best = torch.empty(B, dtype=torch.float64, device=u.device)
        if resume is not None:
            lb_state.copy_(resume["lbfgs_state"])
            u_best.copy_(resume["u_best"])
            F_best.copy_(resume["F_best"])
    elif optimizer != "gd":
        raise ValueError(f"unknown optimizer {optimizer!r}")
    done = it0                                  # iterations completed (evaluation and update)
    for it in range(it0, it0 + iters):
        redo.redo_quantize(table.handle, u, q)
        if state:
            redo.redo_state_grad(table.handle, q, prec, psi0, target, F, g, ws)
        elif drift is not None:
            redo.redo_fidelity_grad_drift(table.handle, q, drift, target, prec, checkpoint_every, F, g, ws,
                                          reunit_every=reunit_every)
        else:
            redo.redo_fidelity_grad(table.handle, q, target, prec, checkpoint_every, F, g, ws,
                                    reunit_every=reunit_every)
        if optimizer == "lbfgs":
            # the accepted point's F (it never falls) is the iteration's fidelity
            redo.redo_grape_lbfgs_step(table.handle, u, g, F, lb_state, it == 0, 8, step, u_best=u_best,
                                       F_best=F_best)
            Fh = F_best.cpu()
            res.F_history.append(Fh.clone())
            res.iterations = done = it + 1
            if on_iter is not None:
                on_iter(it, u, Fh)
            if threshold is not None:
                newly = (Fh >= threshold) & (reached < 0)
                reached[newly] = it
                if bool((reached >= 0).all()):
                    break
            continue
        Fh = F.cpu()
        res.F_history.append(Fh.clone())
        if threshold is not None:
            newly = (Fh >= threshold) & (reached < 0)
            reached[newly] = it
            if bool((reached >= 0).all()):
                break
        if optimizer == "adam":
            redo.redo_grape_adam_step(table.handle, u, g, m_, v_, it + 1, step / (1.0 + it / lr_decay))
            res.iterations = done = it + 1
            if on_iter is not None:
                on_iter(it, u, Fh)
            continue
        if adaptive and prev_F is not None:
            worse = Fh < prev_F
            scale_h = torch.where(worse, scale_h * 0.5, torch.clamp(scale_h * 1.1, max=8.0))
            scale_d.copy_(scale_h, non_blocking=True)
        prev_F = Fh
        redo.redo_grape_step(table.handle, u, g, step, scale_d if adaptive else None)
        res.iterations = done = it + 1
        if on_iter is not None:
            on_iter(it, u, Fh)
    res.u = u_best if optimizer == "lbfgs" else u
    res.reached = reached
    B_ = u.shape[0]
    res.state = {"optimizer": optimizer, "iteration": done, "u": u.clone(), "reached": reached.clone(),
                 # completed iterations only: an iteration stopped by the threshold before its
                 # update is evaluated again on resume
                 "F_history": (torch.stack(res.F_history[:done]) if done > 0
                               else torch.empty((0, B_), dtype=torch.float64)),
                 "scale": scale_h.clone(), "prev_F": None if prev_F is None else prev_F.clone()}
    if optimizer == "adam":
        res.state.update(m=m_.clone(), v=v_.clone())
    elif optimizer == "lbfgs":
        res.state.update(lbfgs_state=lb_state.clone(), u_best=u_best.clone(), F_best=F_best.clone())
    return res
