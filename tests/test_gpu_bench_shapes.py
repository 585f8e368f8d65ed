"""Oracle parity at the launch shapes the benchmark times.

* Batched propagation: N=64 (6 qubits), K=12, B=256 pulses, M=2000 steps, 4096 levels, the
  level table (one operator per control level), split-FP16 tensor-core chains re-unitarised
  every 64 steps -- the benchmark's own call, on all 256 pulses -- with pulses 0, 131 and 255
  checked against the oracle's digit-product chain (max |dU| <= 2e-4, |dF| <= 1e-6), and the
  FP64 and FP32 forms of the same call on those pulses.  FP32: 2e-4.  FP64: a chain of n = 24 000
  operator products (M K d) in which both sides round every product (unit roundoff u = 1.1e-16)
  and use table operators that agree to ~1e-15 (a table entry is reused across the chain, so its
  error adds coherently) drifts apart linearly in n; the bar is n * 8e-16 = 1.9e-11 (the other FP64
  parity tests, with at most a few thousand products, keep 1e-12).
* GRAPE gradient: N=256 (8 qubits), K=16, dt=2 us, the level table filled in closed form,
  every forward state kept, checkpoints every 32 steps, split-FP16 products, at M=64 (the
  benchmark runs M=1000 with the same plan: several checkpoint segments, each run as two
  half segments).  Every entry against the oracle's gradient (1e-3 of the largest, as for the
  other split-FP16 gradients) and 20 entries against central differences of the split model
  (h = 1e-6 in normalised amplitude).
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


def test_level_table_benchmark_launch_matches_oracle():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(1, seed=1, B=256, M=2000)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True, levels=True)
    dev = torch.device("cuda")
    u = torch.tensor(w.u, device=dev)
    q = torch.empty(u.shape, dtype=torch.int32, device=dev)
    st = redo.new_status(dev)
    redo.redo_quantize(t.handle, u, q, st)
    U = torch.empty((w.B, w.N, w.N), dtype=torch.complex128, device=dev)
    F = torch.empty(w.B, dtype=torch.float64, device=dev)
    tau = torch.empty(w.B, dtype=torch.complex128, device=dev)
    target = torch.as_tensor(w.target, device=dev)
    redo.redo_propagate(t.handle, q, "fp16x3", U, target, F, tau, t.workspace(w.B, w.M, "fp16x3", 64), st,
                        reunit_every=64)
    picks = [0, 131, 255]
    qs = q[picks].contiguous()
    sub = {}
    for prec, reunit in (("fp64", 0), ("fp32", 64)):
        Us = torch.empty((3, w.N, w.N), dtype=torch.complex128, device=dev)
        Fs = torch.empty(3, dtype=torch.float64, device=dev)
        redo.redo_propagate(t.handle, qs, prec, Us, target, Fs, None, t.workspace(3, w.M, prec, reunit), st,
                            reunit_every=reunit)
        sub[prec] = (Us.cpu().numpy(), Fs.cpu().numpy())
    torch.cuda.synchronize()
    assert st.cpu().numpy()[2:].tolist() == [0, 0]
    qo, dig, _, _ = _ref.oracle_levels(w, w.u[picks])
    assert np.array_equal(q[picks].cpu().numpy(), qo)
    T, D = _ref.oracle_table(w, method="eig")
    Ug, Fg = U.cpu().numpy(), F.cpu().numpy()
    for i, b in enumerate(picks):
        Uo = O.propagate(T, D, dig[i])
        Fo = O.fidelity(w.target, Uo)
        assert np.abs(Ug[b] - Uo).max() < 2e-4
        assert abs(Fg[b] - Fo) < 1e-6
        assert np.abs(sub["fp64"][0][i] - Uo).max() < w.M * w.K * w.digits * 8e-16
        assert abs(sub["fp64"][1][i] - Fo) < 1e-12
        assert np.abs(sub["fp32"][0][i] - Uo).max() < 2e-4
        assert abs(sub["fp32"][1][i] - Fo) < 1e-6
    t.close()


class _SplitModel:
    """The split model's fidelity with one coefficient moved off its level value, from the
    oracle's step factors with every other step's propagator formed once."""

    def __init__(self, T, D, w, dig, uhat, target):
        self.T, self.D, self.w, self.dig, self.uhat, self.target = T, D, w, dig, uhat, target
        steps = [O.step_propagator(T, D, dig[s]) for s in range(w.M)]
        I = np.eye(w.N, dtype=np.complex128)
        self.prefix = [I]                      # prefix[n] = U_n ... U_1 (0-based steps < n)
        for s in range(w.M):
            self.prefix.append(steps[s] @ self.prefix[-1])
        self.suffix = [I] * (w.M + 1)          # suffix[n] = U_M ... U_{n+1} (0-based steps > n - 1)
        for s in range(w.M - 1, -1, -1):
            self.suffix[s] = self.suffix[s + 1] @ steps[s]

    def fidelity(self, n, k, delta):
        E = O.step_factors(self.T, self.D, self.dig[n])
        E[k] = self.T.factor(k, self.uhat[n, k] + delta)
        Us = self.D
        for Ek in E:
            Us = Ek @ Us
        return O.fidelity(self.target, self.suffix[n + 1] @ Us @ self.prefix[n])


def test_grape_gradient_benchmark_plan_n256_matches_oracle():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(2, M=64)                                # N=256, K=16, dt=2 us, Haar target
    assert (w.N, w.K) == (256, 16)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=False, fp16x3=True, levels=True)
    q = t.quantize(w.u)
    st = redo.new_status()
    F, g = t.fidelity_grad(q, w.target, "fp16x3", checkpoint_every=32, status=st)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[2:].tolist() == [0, 0]
    g = g.cpu().numpy()[0]
    T = _ref.LazyTable(w)
    D = O.expm_hermitian(w.H0, w.dt)
    qo, dig, _, _ = _ref.oracle_levels(w)
    assert np.array_equal(q.cpu().numpy(), qo)
    Fo, go = O.grape_gradient(T, D, w.Hk, w.dt, dig[0], w.target)
    assert abs(F.cpu().numpy()[0] - Fo) < 1e-6
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()
    # central differences of the split model at the level values, 20 random entries
    uhat = O.level_values(qo[0], w.lo, w.hi, w.levels)
    h = 1e-6 * w.extra["Omega"]
    model = _SplitModel(T, D, w, dig[0], uhat, w.target)
    assert abs(model.fidelity(0, 0, 0.0) - Fo) < 1e-12
    rng = np.random.default_rng(8)
    for _ in range(20):
        n, k = int(rng.integers(w.M)), int(rng.integers(w.K))
        fd = (model.fidelity(n, k, h) - model.fidelity(n, k, -h)) / (2 * h)
        # F ~ 1e-5 against a Haar target: rounding of F is ~1e-21, far below these bounds
        assert abs(fd - go[n, k]) <= 1e-6 * np.abs(go).max()
        assert abs(fd - g[n, k]) <= 1e-3 * np.abs(go).max()
    t.close()
