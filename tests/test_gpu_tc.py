"""Tensor-core (tcgen05, split-FP16) chains against the FP64 oracle and the FP64 GPU path.

The split-FP16 path is a reduced-precision form: parity is a bound, not bit
equality -- max-entry error <= 2e-4 on chains of up to 48 000 products and
|dF| <= 1e-6 on the fidelity.
"""
import numpy as np
import pytest
import torch

from oracle import redo_oracle as O
from paper_1707_02162_gb300 import inputs
from tests import _ref

pytestmark = pytest.mark.gpu

TC_TOL = 2e-4
F_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02162_gb300 import build
    build.build()


def _table(w):
    from paper_1707_02162_gb300 import redo
    return redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True)


def _run(w, pulses=None, reunit=64):
    from paper_1707_02162_gb300 import redo
    t = _table(w)
    st = redo.new_status()
    q = t.quantize(w.u, st)
    U, F, _ = t.propagate(q, "fp16x3", target=w.target, status=st, reunit_every=reunit)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[2:].tolist() == [0, 0]
    q_ref, dig, _, _ = _ref.oracle_levels(w)
    T, D = _ref.oracle_table(w)
    pulses = list(range(w.B)) if pulses is None else pulses
    Uo = _ref.oracle_propagators(w, T, D, dig, pulses)
    Ug = U.cpu().numpy()[pulses]
    err = np.abs(Ug - Uo).max()
    Fo = np.array([O.fidelity(w.target, Uo[i]) for i in range(len(pulses))])
    dF = np.abs(F.cpu().numpy()[pulses] - Fo).max()
    return err, dF, t, q


def test_tc_single_short_chain():
    w = inputs.config(1, B=1, M=3)            # 72 factors: one segment
    err, dF, _, _ = _run(w, reunit=0)
    assert err < 1e-5, err
    assert dF < F_TOL


@pytest.mark.parametrize("reunit", [0, 16])
def test_tc_small_batch_ragged(reunit):
    w = inputs.config(1, B=5, M=57)           # 57 steps: ragged against 16-step segments
    err, dF, _, _ = _run(w, reunit=reunit)
    assert err < TC_TOL, err
    assert dF < F_TOL


def test_tc_zero_steps_identity():
    w = inputs.config(1, B=3, M=0)
    t = _table(w)
    q = torch.zeros((3, 0, w.K), dtype=torch.int32, device="cuda")
    U, F, _ = t.propagate(q, "fp16x3", target=w.target)
    assert np.abs(U.cpu().numpy() - np.eye(w.N)).max() == 0


def test_tc_full_size_sampled_against_oracle_and_fp64():
    w = inputs.config(1)                      # B=256, M=2000: the benchmark's launch configuration
    err, dF, t, q = _run(w, pulses=[0, 131, 255])
    assert err < TC_TOL, err
    assert dF < F_TOL, dF
    U16, F16, _ = t.propagate(q, "fp16x3", target=w.target, reunit_every=64)
    U64, F64, _ = t.propagate(q[:8].contiguous(), "fp64", target=w.target)
    assert (U16[:8] - U64).abs().max().item() < TC_TOL
    assert (F16[:8] - F64).abs().max().item() < F_TOL
    # every pulse: unitary to the reduced-precision level
    G = torch.einsum("bji,bjk->bik", U16.conj(), U16)
    eye = torch.eye(w.N, dtype=G.dtype, device=G.device)
    assert (G - eye).abs().max().item() < 1e-10       # re-unitarised in FP64 at the end


def test_tc_without_reunit_drifts_in_norm():
    # documents why the reduced form re-unitarises: without it the FP32
    # accumulation shrinks the chain's singular values
    w = inputs.config(1, B=4, M=2000)
    from paper_1707_02162_gb300 import redo
    t = _table(w)
    q = t.quantize(w.u)
    U0, _, _ = t.propagate(q, "fp16x3", reunit_every=0)
    U1, _, _ = t.propagate(q, "fp16x3", reunit_every=64)
    U64, _, _ = t.propagate(q, "fp64")
    e0 = (U0 - U64).abs().max().item()
    e1 = (U1 - U64).abs().max().item()
    assert e1 < e0 and e1 < TC_TOL


def test_tc_requires_planes():
    from paper_1707_02162_gb300 import redo
    w = inputs.config(1, B=1, M=2)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=False)
    q = t.quantize(w.u)
    with pytest.raises(redo.RedoError):
        t.propagate(q, "fp16x3")


def test_tc_level_table_matches_oracle():
    # process 3: every level's operator evaluated once; a step costs K products
    from paper_1707_02162_gb300 import redo
    w = inputs.config(1, B=4, M=120)
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True, levels=True)
    assert t.info["digits"] == 1 and t.info["base"] == w.levels and t.info["entries"] == w.K * w.levels
    q = t.quantize(w.u)
    U, F, _ = t.propagate(q, "fp16x3", target=w.target, reunit_every=64)
    U64, F64, _ = t.propagate(q, "fp64", target=w.target)
    T, D = _ref.oracle_table(w)
    _, dig, _, _ = _ref.oracle_levels(w)
    Uo = _ref.oracle_propagators(w, T, D, dig, range(w.B))
    assert np.abs(U64.cpu().numpy() - Uo).max() < 1e-12
    assert np.abs(U.cpu().numpy() - Uo).max() < TC_TOL
    assert (F - F64).abs().max().item() < F_TOL


@pytest.mark.parametrize("variant", ["1", "2", "3"])
def test_tc_kernel_variants_match(monkeypatch, variant):
    # 1: state operand in shared memory (embedding), 2: in tensor memory,
    # 3 (default): three-block state in shared memory
    from paper_1707_02162_gb300 import redo
    w = inputs.config(1, B=7, M=80)                 # 7 pulses: a ragged last CTA for 2 and 3 chains
    t = redo.Table(w.H0, w.Hk, w.dt, w.lo, w.hi, w.base, w.digits, fp32=True, fp16x3=True, levels=True)
    q = t.quantize(w.u)
    monkeypatch.setenv("REDO_TC_VARIANT", "1")
    U1, F1, _ = t.propagate(q, "fp16x3", target=w.target, reunit_every=16)
    monkeypatch.setenv("REDO_TC_VARIANT", variant)
    U2, F2, _ = t.propagate(q, "fp16x3", target=w.target, reunit_every=16)
    U3, _, _ = t.propagate(q, "fp16x3", reunit_every=0)
    monkeypatch.delenv("REDO_TC_VARIANT")
    U64, _, _ = t.propagate(q, "fp64")
    assert (U2 - U64).abs().max().item() < TC_TOL
    assert (U3 - U64).abs().max().item() < TC_TOL
    assert (U1 - U2).abs().max().item() < TC_TOL
    assert (F1 - F2).abs().max().item() < F_TOL
