"""Learned warm start: GPU MLP kernels against the FP64 oracle, and the gain of
an MLP-initialised REDO-GRAPE over random initialisation on a reachable
single-qubit family of targets."""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


@pytest.mark.parametrize("sizes,batch", [([23, 64, 64, 64, 100], 8), ([5, 33, 17, 70], 65),
                                         ([23, 512, 512, 512, 5000], 200)])
def test_mlp_forward_backward_match_oracle(sizes, batch):
    # The GEMMs are split-BF16 tensor-core products: an operand v is carried as hi + lo with
    # |v - hi - lo| <= 2^-16 |v| (bf16 keeps 8 significant bits), and a product drops lo*lo'
    # (<= 2^-16 |a b|), so every term of a sum is exact to 3 * 2^-16 = 4.6e-5 of itself; the
    # FP32 accumulation adds ~2^-24 per addition.  Term errors of random sign add like a random
    # walk, so a sum -- and, layer after layer, each gradient -- stays within about the per-term
    # bound of its own size (measured on a GB300: 3.6e-6 absolute on outputs in [-1, 1], 1.7e-5
    # of the largest gradient entry).  Bars: outputs 2e-5, gradients 1e-4 of their largest entry.
    from paper_1707_02162_gb300.warmstart import MLP
    from paper_1707_02162_gb300 import redo
    rng = np.random.default_rng(0)
    params = O.mlp_init(sizes, rng)
    for W, b in params:
        b[:] = rng.uniform(-0.1, 0.1, size=b.shape)
    x = rng.standard_normal((batch, sizes[0]))
    yt = rng.uniform(-1, 1, size=(batch, sizes[-1]))
    y_o, cache = O.mlp_forward(params, x)
    loss_o, grads_o = O.mlp_backward(params, cache, yt)
    net = MLP(sizes, params=_flat(params))
    y = net.forward(torch.tensor(x)).cpu().numpy()
    assert np.abs(y - y_o).max() < 2e-5
    _, na, nw = redo.redo_mlp_sizes(sizes, batch)
    acts = torch.empty(na, dtype=torch.float32, device="cuda")
    work = torch.empty(nw, dtype=torch.float32, device="cuda")
    yy = torch.empty((batch, sizes[-1]), dtype=torch.float32, device="cuda")
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    redo.redo_mlp_forward(sizes, net.params, xt, acts, yy)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    redo.redo_mlp_backward(sizes, net.params, xt, acts, torch.tensor(yt, dtype=torch.float32, device="cuda"),
                           net.grads, loss, work)
    g = net.grads.cpu().numpy()
    go = _flat(grads_o)
    assert abs(loss.item() - loss_o) < 1e-5 * max(1.0, loss_o)
    assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()


def test_adam_matches_oracle():
    from paper_1707_02162_gb300 import redo
    rng = np.random.default_rng(1)
    p = rng.standard_normal(1000)
    g = rng.standard_normal(1000)
    m = np.zeros(1000)
    v = np.zeros(1000)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    mt, vt = torch.zeros_like(pt), torch.zeros_like(pt)
    for step in range(1, 4):
        gt = torch.tensor(g * step, dtype=torch.float32, device="cuda")
        redo.redo_mlp_adam(pt, gt, mt, vt, step, 1e-2)
        p, m, v = O.adam_step(p, g * step, m, v, step, 1e-2)
    assert np.abs(pt.cpu().numpy() - p).max() < 1e-5


def _single_qubit_family(n_inst, seed):
    """Targets exp(-i (t1 X + t2 Y + t3 Z)), t ~ U[0, pi/4]; one qubit with a small offset."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0, np.pi / 4, size=(n_inst, 3))
    targets = np.stack([O.expm_hermitian(inputs.pauli_generator(["X", "Y", "Z"], th), 1.0) for th in theta])
    return theta, targets


def test_warm_start_beats_random_init():
    from paper_1707_02162_gb300 import redo
    from paper_1707_02162_gb300.warmstart import MLP, converge
    Om = 2 * np.pi * 1e4
    H0 = 2 * np.pi * 800.0 * inputs.PAULI["Z"] / 2
    Hk = np.stack([inputs.PAULI["X"] / 2, inputs.PAULI["Y"] / 2])
    M, dt, K = 40, 2e-6, 2
    t = redo.Table(H0, Hk, dt, np.full(K, -Om), np.full(K, Om), 64, 2, fp32=True)
    thr, step = 0.999, 3e9
    th_tr, T_tr = _single_qubit_family(192, 11)
    rng = np.random.default_rng(2)
    u0 = rng.uniform(-0.3 * Om, 0.3 * Om, size=(192, M, K))
    u_tr, reached_tr, _ = converge(t, T_tr, u0, 400, step, thr)
    ok = np.array(reached_tr) >= 0
    assert ok.mean() > 0.8
    # train on converged pulses (normalised amplitude), features = angles scaled to [-1, 1]
    feats = torch.tensor(th_tr[ok] / (np.pi / 8) - 1.0, dtype=torch.float32)
    targ = torch.tensor(u_tr.cpu().numpy()[ok].reshape(ok.sum(), -1) / Om, dtype=torch.float32)
    net = MLP([3, 128, 128, 128, M * K], seed=3)
    loss0 = None
    for it in range(1500):
        loss = net.train_step(feats, targ, 2e-3)
        loss0 = loss if loss0 is None else loss0
    assert loss < 0.2 * loss0
    th_te, T_te = _single_qubit_family(32, 99)
    u_mlp = net.forward(torch.tensor(th_te / (np.pi / 8) - 1.0)).cpu().numpy().reshape(32, M, K) * Om
    u_rnd = np.random.default_rng(5).uniform(-0.3 * Om, 0.3 * Om, size=(32, M, K))
    _, it_mlp, _ = converge(t, T_te, u_mlp.astype(np.float64), 400, step, thr)
    _, it_rnd, _ = converge(t, T_te, u_rnd, 400, step, thr)
    med = lambda v: np.median([x if x >= 0 else 10 ** 6 for x in v])
    assert med(it_mlp) < med(it_rnd)
