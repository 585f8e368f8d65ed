"""Mixed diagonal-state expectations (Tr[rho(t) O]) and the noisy exotic-freezing order
parameter of Section IV on the GPU, against the oracle's dense-matrix definition."""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs

pytestmark = pytest.mark.gpu

H0_AMP = inputs.FREEZE_H0_AMP


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _gpu_table(M, T):
    from paper_1707_02162_gb300 import redo
    H0, Hk, rho, obs = inputs.freezing_system(3, H0_AMP, basis="x")
    t = redo.Table(H0, Hk, T / M, np.array([-H0_AMP]), np.array([H0_AMP]), 100, 2, fp32=True)
    return t, rho, obs


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_freezing_series_matches_oracle(prec, tol):
    M, T = 300, 2 * np.pi
    u = inputs.freezing_drive([7.0, 13.06], [0.0, 0.4], M, T=T)
    t, rho, obs = _gpu_table(M, T)
    q = t.quantize(u)
    ex, mean = t.expect_diag(q, rho, obs, prec)
    H0z, Hkz, rho0, obsz = inputs.freezing_system(3, H0_AMP, basis="z")
    lo, hi = np.array([-H0_AMP]), np.array([H0_AMP])
    To, Do = O.build_table(H0z, Hkz, T / M, lo, hi, 10000, 100, 2)
    qo, _, _ = O.quantize(u, lo, hi, 10000)
    dig = O.level_digits(qo, 100, 2)
    exg = ex.cpu().numpy()
    for b in range(u.shape[0]):
        eo, _ = O.expect_mixed(To, Do, dig[b], rho0, obsz)
        assert np.abs(exg[b] - eo).max() < tol * abs(eo[0])
        assert abs(mean.cpu().numpy()[b] - exg[b, 1:].mean()) < 1e-12 * abs(eo[0])


def test_freezing_at_first_bessel_root_gpu():
    M = 10000
    w1 = 2 * H0_AMP / 2.404825557695773
    u = inputs.freezing_drive([w1 - 3.0, w1, w1 + 3.0], [0.0], M)
    t, rho, obs = _gpu_table(M, inputs.FREEZE_T)
    q = t.quantize(u)
    _, mean = t.expect_diag(q, rho, obs, "fp32", series=False)
    Q = mean.cpu().numpy() / float(np.sum(rho * obs))
    assert Q[1] > 0.99 and Q[1] > Q[0] + 0.1 and Q[1] > Q[2] + 0.1


@pytest.mark.parametrize("n,B,prec,tol", [(1, 3, "fp64", 1e-12), (4, 3, "fp64", 1e-12), (4, 3, "fp32", 2e-5),
                                         (1, 19461, "fp32", 2e-5), (3, 4870, "fp64", 1e-12),
                                         (3, 4870, "fp32", 2e-5), (4, 2450, "fp32", 2e-5)])
def test_expect_diag_random_diagonals(n, B, prec, tol):
    # generic diagonal rho and O on the x/y-controlled ZZ system, N = 2 .. 16; the large batches
    # take the column-per-thread kernel (N <= 16 in FP32, <= 8 in FP64; at least one CTA of
    # 256 / N pulses per SM) with idle lanes in its last CTA, the small ones the CTA-per-pulse
    # kernel
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, n_qubits=n, B=B, M=25, base=16, digits=2)
    rng = np.random.default_rng(9)
    rho, obs = rng.uniform(-1, 1, w.N), rng.uniform(-1, 1, w.N)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True)
    ex, mean = t.expect_diag(t.quantize(w.u), rho, obs, prec)
    To, Do = O.build_table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.levels, w.base, w.digits)
    qo, _, _ = O.quantize(w.u, w.lo, w.hi, w.levels)
    dig = O.level_digits(qo, w.base, w.digits)
    for b in sorted({0, 1, w.B // 2, w.B - 2, w.B - 1}):
        Tf = To.copy()
        eo, _ = O.expect_mixed(Tf, Do, dig[b], np.diag(rho).astype(complex), np.diag(obs).astype(complex))
        assert np.abs(ex.cpu().numpy()[b] - eo).max() < tol
        assert abs(mean.cpu().numpy()[b] - eo[1:].mean()) < tol


def test_expect_diag_rejects_unsupported():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(0, n_qubits=7, B=1, M=4, base=16, digits=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits)
    with pytest.raises(redo.RedoError):
        t.expect_diag(t.quantize(w.u), np.ones(128), np.ones(128), "fp64")


def test_expect_diag_zero_steps_mean_is_initial_value():
    t, rho, obs = _gpu_table(10, 1.0)
    q = torch.zeros((3, 0, 1), dtype=torch.int32, device="cuda")
    ex, mean = t.expect_diag(q, rho, obs, "fp64")
    assert ex.shape == (3, 1)
    assert np.abs(ex.cpu().numpy()[:, 0] - np.sum(rho * obs)).max() < 1e-12
    assert np.abs(mean.cpu().numpy() - np.sum(rho * obs)).max() < 1e-12
