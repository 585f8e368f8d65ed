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


def test_plain_n8_replicas_sampled_against_oracle():
    """The plain-REDO key: 3 qubits, M=1000, 4096 replica pulses, FP64 and FP32, in one call each;
    three sampled pulses against the oracle, unitarity and F in [0, 1] for every pulse."""
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, B=4096)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    q = t.quantize(w.u)
    picks = [0, 2047, 4095]
    qo, dig, _, _ = _ref.oracle_levels(w, w.u[picks])
    assert np.array_equal(q[picks].cpu().numpy(), qo)
    T, D = _ref.oracle_table(w)
    Uo = np.stack([O.propagate(T, D, dig[i]) for i in range(len(picks))])
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-4)):
        U, F, _ = t.propagate(q, prec, target=w.target)
        Ug, Fg = U.cpu().numpy(), F.cpu().numpy()
        assert np.abs(Ug[picks] - Uo).max() < tol
        for i, b in enumerate(picks):
            assert abs(Fg[b] - O.fidelity(w.target, Uo[i])) < (1e-12 if prec == "fp64" else 1e-6)
        G = np.einsum("bji,bjk->bik", Ug.conj(), Ug)
        assert np.abs(G - np.eye(w.N)).max() < (1e-12 if prec == "fp64" else 1e-4)
        assert ((Fg >= 0) & (Fg <= 1 + 1e-9)).all()
    t.close()


def test_warm_start_batched_drift_gradient_sampled_against_oracle():
    """The batched warm-start GRAPE call: N=32, K=10, M=500, 256 instances each with its own
    diagonal drift, FP32 chains with every forward state kept; three instances against the oracle."""
    from paper_1707_02162_gb300 import redo
    w = inputs.config(4, B=256)
    h = inputs.drift_diagonals(w)
    rng = np.random.default_rng(0)
    targets = np.stack([inputs.haar_unitary(rng, w.N) for _ in range(w.B)])
    t = redo.Table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    q = t.quantize(w.u)
    F, g = t.fidelity_grad_drift(q, h, targets, "fp32")
    picks = [0, 128, 255]
    T, _ = O.build_table(np.zeros_like(w.H0), w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits, method="eig")
    qo, dig, _, _ = _ref.oracle_levels(w, w.u[picks])
    assert np.array_equal(q[picks].cpu().numpy(), qo)
    for i, b in enumerate(picks):
        Db = O.expm_hermitian(np.diag(h[b]).astype(np.complex128), w.dt)
        Fo, go = O.grape_gradient(T, Db, w.Hk, w.dt, dig[i], targets[b])
        assert abs(F.cpu().numpy()[b] - Fo) < 1e-6
        assert np.abs(g.cpu().numpy()[b] - go).max() <= 2e-4 * np.abs(go).max()
    t.close()


def test_ensemble_n1024_full_length_properties():
    """The N=1024 ensemble key at full length (64 realisations x 2000 steps, level table, split
    FP16 propagators and the FP32 state path), checked through properties and the FP64 path, as
    the oracle cannot run 2000 products of 1024 x 1024 operators per realisation here:
      * <Z_1>(t) of the reduced path against the FP64 state path (|d| <= 1e-4), and 1 at t = 0;
      * the final propagator of one realisation against the FP64 propagator; without
        re-unitarisation the split-FP16 chain loses norm coherently (~4e-6 per 1024 x 1024
        product, so U^dag U = (1 - 0.008) I after 2000), bounded below 2e-2, and every entry
        (modulus <= 1) moves by at most half that beyond the 5e-4 rounding bar;
      * <Z_1> at the last step recomputed from the propagator's first column (U |0...0>);
      * with reunit_every = 500 the same propagator is unitary to 1e-4."""
    from paper_1707_02162_gb300 import redo
    w = inputs.config(3)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=False, fp16x3=True, levels=True)
    q = t.quantize(w.u)
    e16, U = t.simulate(q, w.psi0, w.obs_diag, "fp16x3", want_U=True)
    e64, _ = t.simulate(q, w.psi0, w.obs_diag, "fp64", want_U=False)
    e16, e64 = e16.cpu().numpy(), e64.cpu().numpy()
    assert e16.shape == (w.B, w.M + 1)
    assert np.abs(e16 - e64).max() < 1e-4
    assert np.abs(e16[:, 0] - 1.0).max() < 1e-6             # <Z_1> of |0...0> before any step
    q0 = q[:1].contiguous()
    _, U64 = t.simulate(q0, w.psi0, w.obs_diag, "fp64", want_U=True)
    U0, U64 = U[0].cpu().numpy(), U64[0].cpu().numpy()
    # FP64: each of the n = 2000 products moves the norm by up to N u (length-N inner products,
    # u = 1.1e-16), coherently along the diagonal, so the bar is n N u = 2.3e-10, doubled.
    assert np.abs(U64.conj().T @ U64 - np.eye(w.N)).max() < 2 * w.M * w.N * 1.12e-16
    drift = np.abs(np.diag(U0.conj().T @ U0) - 1.0).max()
    assert drift < 2e-2
    assert np.abs(U0 - U64).max() < 5e-4 + drift           # |entries| <= 1 lose at most drift / 2
    for b in (0, 31, 63):
        Ub = U[b].cpu().numpy()
        db = np.abs(np.diag(Ub.conj().T @ Ub) - 1.0).max()
        assert db < 2e-2
        col = Ub[:, 0]                                       # U |0...0>
        assert abs(float(np.sum(w.obs_diag * np.abs(col) ** 2)) - e64[b, -1]) < 2 * db + 1e-4
    _, Ur = t.simulate(q0, w.psi0, w.obs_diag, "fp16x3", reunit_every=500, want_U=True)
    Ur = Ur[0].cpu().numpy()
    assert np.abs(Ur.conj().T @ Ur - np.eye(w.N)).max() < 1e-4
    assert np.abs(Ur - U64).max() < 5e-4
    t.close()
