"""GRAPE by projected L-BFGS on the GPU against the oracle's L-BFGS step.

* ``redo_grape_lbfgs_step`` step by step against ``O.grape_lbfgs_step`` on concave quadratics
  (one per pulse, with a first step large enough to be rejected and backtracked), both sides fed
  the same evaluated point every step: the next trial points agree to 1e-10 of the grid span and
  the accepted fidelities are identical.  Per-pulse sizes of 120 and 700 coefficients (less and
  more than the CTA's 256 threads).
* The device loop ``grape(optimizer="lbfgs")`` against the same loop driven by the oracle's
  gradient and L-BFGS step on an N=8 system: accepted F to 1e-12 and coefficients to 1e-9 of the
  grid width for ten iterations.
* On a reachable target the L-BFGS loop gets past F = 0.999 in fewer evaluations than Adam.
"""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs
from tests import _ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _table(w):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)


@pytest.mark.parametrize("M,K", [(40, 3), (70, 10)])
def test_lbfgs_kernel_steps_match_oracle(M, K):
    from paper_1707_02162_gb300 import redo
    w = inputs.config(4 if K == 10 else 0, B=1, M=4)
    if K == 3:
        w.Hk = np.concatenate([w.Hk, w.Hk[:1]])
        w.lo, w.hi = np.append(w.lo, -3e4), np.append(w.hi, 2e4)
    assert w.Hk.shape[0] == K
    t = _table(w)
    B, n = 4, M * K
    rng = np.random.default_rng(M + K)
    span = 0.5 * (w.hi - w.lo).max()
    mats, centres = [], []
    for b in range(B):
        A = rng.standard_normal((n, n)) / np.sqrt(n)
        mats.append((A @ A.T + 0.2 * np.eye(n)) / span ** 2)
        centres.append(rng.uniform(w.lo, w.hi, size=(M, K)) * 0.5)

    def Fg(b, u):
        e = (u - centres[b]).ravel()
        return -0.5 * e @ mats[b] @ e, -(mats[b] @ e).reshape(M, K)

    u = np.stack([rng.uniform(w.lo, w.hi, size=(M, K)) for _ in range(B)])
    ud = torch.tensor(u, device="cuda")
    gd = torch.empty_like(ud)
    Fd = torch.empty(B, dtype=torch.float64, device="cuda")
    Fbest = torch.empty_like(Fd)
    state = torch.empty(redo.redo_grape_lbfgs_workspace(t.handle, B, M, 5), dtype=torch.uint8, device="cuda")
    ostate = [{} for _ in range(B)]
    rejected = 0
    F0 = [Fg(b, u[b])[0] for b in range(B)]
    for it in range(25):
        cur = ud.cpu().numpy()
        FG = [Fg(b, cur[b]) for b in range(B)]
        gd.copy_(torch.tensor(np.stack([g for _, g in FG])))
        Fd.copy_(torch.tensor([F for F, _ in FG]))
        redo.redo_grape_lbfgs_step(t.handle, ud, gd, Fd, state, it == 0, history=5, step0=0.9, F_best=Fbest)
        nxt = ud.cpu().numpy()
        Fb = Fbest.cpu().numpy()
        for b in range(B):
            before = ostate[b].get("F")
            un, ostate[b] = O.grape_lbfgs_step(cur[b], FG[b][1], FG[b][0], ostate[b], w.lo, w.hi, history=5,
                                               step0=0.9, first=(it == 0))
            rejected += int(before is not None and ostate[b]["F"] == before)
            assert np.abs(nxt[b] - un).max() <= 1e-10 * span
            assert Fb[b] == ostate[b]["F"]
    assert rejected > 0                                     # backtracking was exercised
    assert all(ostate[b]["F"] > 1e-2 * F0[b] for b in range(B))   # and the ascent closed on the maximum (F = 0)
    t.close()


def test_lbfgs_grape_loop_matches_oracle_loop():
    from paper_1707_02162_gb300.grape import grape
    w = inputs.config(0, B=2, M=24)
    w.target = inputs.haar_unitary(np.random.default_rng(11), w.N)
    t = _table(w)
    T, D = _ref.oracle_table(w)
    seen = []
    grape(t, w.target, torch.tensor(w.u, device="cuda"), iters=10, step=0.05, prec="fp64", optimizer="lbfgs",
          on_iter=lambda it, u, F: seen.append((u.cpu().numpy().copy(), F.numpy().copy())))
    u = w.u.copy()
    states = [{} for _ in range(w.B)]
    width = (w.hi - w.lo).max()
    for it in range(10):
        q, _, _ = O.quantize(u, w.lo, w.hi, w.levels)
        dig = O.level_digits(q, w.base, w.digits)
        for b in range(w.B):
            F, g = O.grape_gradient(T, D, w.Hk, w.dt, dig[b], w.target)
            u[b], states[b] = O.grape_lbfgs_step(u[b], g, F, states[b], w.lo, w.hi, history=8, step0=0.05,
                                                 first=(it == 0))
        assert np.abs(seen[it][1] - np.array([s["F"] for s in states])).max() < 1e-12
        assert np.abs(seen[it][0] - u).max() <= 1e-9 * width
    t.close()


def test_lbfgs_reaches_a_reachable_target_sooner_than_adam():
    from paper_1707_02162_gb300 import redo
    from paper_1707_02162_gb300.grape import grape
    w = inputs.config(0, B=4, M=60)
    t = _table(w)
    # targets: the propagators of other pulses on the same grid (reachable by construction)
    rng = np.random.default_rng(21)
    other = rng.uniform(w.lo[0], w.hi[0], size=w.u.shape)
    U, _, _ = t.propagate(t.quantize(other), "fp64")
    targets = U
    u0 = torch.tensor(rng.uniform(w.lo[0], w.hi[0], size=w.u.shape) * 0.3, device="cuda")
    r_lb = grape(t, targets, u0, iters=300, step=0.05, prec="fp64", optimizer="lbfgs", threshold=0.999)
    r_ad = grape(t, targets, u0, iters=300, step=0.01 * w.extra["Omega"], prec="fp64", optimizer="adam",
                 threshold=0.999)
    assert (r_lb.reached >= 0).all()
    it_lb = r_lb.reached.double().median().item()
    it_ad = torch.where(r_ad.reached >= 0, r_ad.reached, torch.tensor(300)).double().median().item()
    assert it_lb < it_ad
    # the returned pulses have the fidelity the loop reports
    Fr = redo.Table.fidelity_grad(t, t.quantize(r_lb.u), targets, "fp64")[0]
    assert (Fr.cpu() >= 0.999).all()
    t.close()
