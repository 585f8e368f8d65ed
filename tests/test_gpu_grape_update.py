"""GRAPE control update on the GPU (Section III, Fig. fc) against the oracle's update.

* ``redo_grape_step`` and ``redo_grape_adam_step`` element by element against
  ``O.grape_update`` / ``O.grape_adam_update`` on arrays that span many blocks of the
  grid-stride loop with a ragged tail, with clipping active at both ends.  The kernels
  contract ``u + s g`` into one fused multiply-add where the oracle rounds twice, so each
  entry may differ by a couple of units in the last place of the larger of the two terms.
* The device-resident loop ``grape()`` (quantize, fidelity + gradient, update; five
  iterations, both optimisers) against the same loop driven by the oracle's gradient and
  update: level indices bit-exact and coefficients within 1e-9 of the grid width after
  every iteration.  The FP64 gradients agree to ~1e-10 of their largest entry, which moves
  a coefficient by far less than that.
"""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs
from tests import _ref

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _table(w):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)


def _grid_case(B=7, M=6007, K=10, seed=21):
    # K=10 terms with different grids; 420 490 coefficients: more than the 152 x 8 x 256
    # threads of one grid-stride pass, not a multiple of the block size
    w = inputs.config(4, B=1, M=4)
    rng = np.random.default_rng(seed)
    lo = -rng.uniform(1e4, 7e4, size=K)
    hi = rng.uniform(1e4, 7e4, size=K)
    w.lo, w.hi = lo, hi
    u = rng.uniform(lo, hi, size=(B, M, K))
    g = rng.standard_normal((B, M, K)) * 1e-7
    return w, u, g


def test_grape_step_kernel_matches_oracle_update():
    from paper_1707_02162_gb300 import redo
    w, u, g = _grid_case()
    t = _table(w)
    B = u.shape[0]
    scale = np.random.default_rng(2).uniform(0.1, 4.0, size=B)
    for step in (3e9, 1e14):                      # the second drives every entry onto a grid end
        ud = torch.tensor(u, device="cuda")
        redo.redo_grape_step(t.handle, ud, torch.tensor(g, device="cuda"), step,
                             torch.tensor(scale, device="cuda"))
        uo = O.grape_update(u, g, step, scale, w.lo, w.hi)
        got = ud.cpu().numpy()
        bound = 4 * ULP * (np.abs(u) + np.abs(step * scale[:, None, None] * g))
        assert (np.abs(got - uo) <= bound).all()
        if step == 1e14:
            at_end = (uo == w.lo) | (uo == w.hi)
            assert at_end.mean() > 0.99
            assert (np.abs(got - uo)[at_end] <= 4 * ULP * np.abs(uo)[at_end]).all()
    # no step factors: every pulse steps by `step`
    ud = torch.tensor(u, device="cuda")
    redo.redo_grape_step(t.handle, ud, torch.tensor(g, device="cuda"), 3e9, None)
    uo = O.grape_update(u, g, 3e9, None, w.lo, w.hi)
    assert (np.abs(ud.cpu().numpy() - uo) <= 4 * ULP * (np.abs(u) + np.abs(3e9 * g))).all()
    t.close()


def test_grape_adam_kernel_matches_oracle_three_steps():
    from paper_1707_02162_gb300 import redo
    w, u, _ = _grid_case(B=3, M=4099, K=10, seed=5)
    t = _table(w)
    rng = np.random.default_rng(6)
    ud = torch.tensor(u, device="cuda")
    md, vd = torch.zeros_like(ud), torch.zeros_like(ud)
    lr = 2e3
    b1, b2 = 0.9, 0.999
    for step in (1, 2, 3):
        g = rng.standard_normal(u.shape) * 1e-7
        g[0, :5] = 0.0                             # zero gradients stay put (eps guards the division)
        # each step is compared from the same state: the kernel's moments and coefficients so far
        u_prev, m_prev, v_prev = ud.cpu().numpy(), md.cpu().numpy(), vd.cpu().numpy()
        redo.redo_grape_adam_step(t.handle, ud, torch.tensor(g, device="cuda"), md, vd, step, lr)
        uo, mo, vo = O.grape_adam_update(u_prev, g, m_prev, v_prev, step, lr, w.lo, w.hi)
        # b1 m + (1 - b1) g can cancel: bound by the size of its terms, not of the result
        assert (np.abs(md.cpu().numpy() - mo) <= 4 * ULP * (b1 * np.abs(m_prev) + (1 - b1) * np.abs(g))).all()
        assert (np.abs(vd.cpu().numpy() - vo) <= 4 * ULP * (b2 * v_prev + (1 - b2) * g * g)).all()
        # |lr * m_hat / (sqrt(v_hat) + eps)| <= lr * (a few), so a few ulps of |u| + lr
        bound = 16 * ULP * (np.abs(u_prev) + lr * 10)
        assert (np.abs(ud.cpu().numpy() - uo) <= bound).all()
    assert np.array_equal(ud.cpu().numpy()[0, :5], u[0, :5])
    t.close()


@pytest.mark.parametrize("optimizer,step", [("gd", 2e10), ("adam", 3e3)])
def test_grape_loop_matches_oracle_loop(optimizer, step):
    from paper_1707_02162_gb300.grape import grape
    w = inputs.config(0, B=3, M=24)                       # N=8, K=2
    w.target = inputs.haar_unitary(np.random.default_rng(11), w.N)
    t = _table(w)
    T, D = _ref.oracle_table(w)
    iters = 5
    seen = []

    def on_iter(it, u, F):
        seen.append((u.cpu().numpy().copy(), F.numpy().copy()))

    res = grape(t, w.target, torch.tensor(w.u, device="cuda"), iters=iters, step=step, prec="fp64",
                optimizer=optimizer, on_iter=on_iter)
    assert res.iterations == iters and len(seen) == iters
    # the same loop with the oracle's arithmetic
    u = w.u.copy()
    scale, F_prev = np.ones(w.B), None
    m, v = np.zeros_like(u), np.zeros_like(u)
    width = (w.hi - w.lo).max()
    for it in range(iters):
        q, _, _ = O.quantize(u, w.lo, w.hi, w.levels)
        dig = O.level_digits(q, w.base, w.digits)
        Fg = [O.grape_gradient(T, D, w.Hk, w.dt, dig[b], w.target) for b in range(w.B)]
        F = np.array([f for f, _ in Fg])
        g = np.stack([gb for _, gb in Fg])
        assert np.abs(seen[it][1] - F).max() < 1e-12
        if optimizer == "adam":
            u, m, v = O.grape_adam_update(u, g, m, v, it + 1, step / (1.0 + it / 150.0), w.lo, w.hi)
        else:
            scale = O.grape_step_scale(scale, F, F_prev)
            F_prev = F
            u = O.grape_update(u, g, step, scale, w.lo, w.hi)
        ug = seen[it][0]
        assert np.abs(ug - u).max() <= 1e-9 * width
        qg, _, _ = O.quantize(ug, w.lo, w.hi, w.levels)
        qo, _, _ = O.quantize(u, w.lo, w.hi, w.levels)
        assert np.array_equal(qg, qo)
    assert seen[-1][1].mean() > seen[0][1].mean()
    t.close()
