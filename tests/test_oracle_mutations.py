"""Planted mistakes in the oracle, each caught by a pin (CPU only).

Every case installs, for the duration of that case only, a variant of one oracle function with
one plausible mistake: a dropped term or factor, a wrong sign, a swapped or reversed order, an
off-by-one index or level, a missing clamp, a lost bias correction.  At least one of the pins
named beside the case must then fail.  The variants are written here from each function's
definition (most wrap the correct function and change one thing about its inputs or outputs);
the oracle module itself is never edited, and ``monkeypatch`` restores it after each case.
"""
import math

import numpy as np
import pytest

from oracle import redo_oracle as O
from tests import test_oracle_pins as P


# ------------------------------------------------------------------ variants written out here

def _quantize_ties_away(u, lo, hi, levels):
    # nearest grid point, but exact ties rounded away from the lower level
    u = np.asarray(u, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    delta = (np.asarray(hi, dtype=np.float64) - lo) / (levels - 1)
    with np.errstate(all="ignore"):
        r = np.floor((u - lo) / delta + 0.5)
    finite = np.isfinite(u)
    sat = finite & ((r < 0) | (r > levels - 1))
    r = np.where(finite, np.clip(np.nan_to_num(r), 0, levels - 1), 0)
    return r.astype(np.int32), int((~finite).sum()), int(sat.sum())


def _grape_update_no_clip(u, g, step, scale, lo, hi):
    s = np.ones(np.asarray(u).shape[0]) if scale is None else np.asarray(scale, dtype=np.float64)
    return np.asarray(u, dtype=np.float64) + step * s[:, None, None] * g


def _adam_no_bias_correction(u, g, m, v, t, lr, lo, hi, beta1=0.9, beta2=0.999, eps=1e-12):
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    x = np.asarray(u, dtype=np.float64) + lr * m / (np.sqrt(v) + eps)
    return np.clip(x, lo, hi), m, v


def _adam_step_no_bias_correction(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    return p - lr * m / (np.sqrt(v) + eps), m, v


def _polar_inverse_not_root(P_):
    P_ = np.asarray(P_, dtype=np.complex128)
    return P_ @ np.linalg.inv(P_.conj().T @ P_)


def _polar_wrong_side(P_):
    # (P^dag P)^(-1/2) P: the inverse root of the Gram matrix applied from the left
    P_ = np.asarray(P_, dtype=np.complex128)
    w, V = np.linalg.eigh(P_.conj().T @ P_)
    return ((V * (1.0 / np.sqrt(w))[None, :]) @ V.conj().T) @ P_


def _split_step_drift_last(H0, Hk, dt, u_row):
    U = np.eye(np.asarray(H0).shape[0], dtype=np.complex128)
    for k in range(Hk.shape[0]):
        U = O.expm_pade13(-1j * dt * u_row[k] * Hk[k]) @ U
    return O.expm_pade13(-1j * dt * np.asarray(H0, dtype=np.complex128)) @ U


def _expect_mixed_one_sided(T, D, digits_bm, rho0, obs):
    # rho(t) = X rho0 with the conjugating X^dag dropped
    N = D.shape[0]
    X = np.eye(N, dtype=np.complex128)
    out = [float(np.trace(rho0 @ obs).real)]
    for n in range(digits_bm.shape[0]):
        X = O.step_propagator(T, D, digits_bm[n]) @ X
        out.append(float(np.trace(X @ rho0 @ obs).real))
    return np.array(out), X


def _gelu_tanh_form(x):
    return 0.5 * x * (1.0 + np.tanh(math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)))


def _gelu_grad_no_density_term(x):
    v = np.vectorize(math.erf, otypes=[np.float64])
    return 0.5 * (1.0 + v(x / math.sqrt(2.0)))


def _mlp_forward_gelu_output(params, x):
    # the output layer through GELU as well, instead of tanh
    h = np.asarray(x, dtype=np.float64)
    cache = [h]
    for W, b in params:
        z = h @ W.T + b
        cache.append(z)
        h = O.gelu(z)
        cache.append(h)
    return h, cache


def _mlp_forward_no_bias(params, x):
    h = np.asarray(x, dtype=np.float64)
    cache = [h]
    for li, (W, _) in enumerate(params):
        z = h @ W.T
        cache.append(z)
        h = np.tanh(z) if li == len(params) - 1 else O.gelu(z)
        cache.append(h)
    return h, cache


def _phase_split_step_no_inverse(H0, Sx, sz, dt, amp_row, phi_row):
    # Z_n E ... E D: the turn back about z (Z_n^dag) dropped
    Zd = np.diag(O.phase_rotation(phi_row, sz))
    E = np.eye(np.asarray(H0).shape[0], dtype=np.complex128)
    for k in range(Sx.shape[0]):
        E = O.expm_pade13(-1j * dt * amp_row[k] * Sx[k]) @ E
    return Zd @ E @ O.expm_pade13(-1j * dt * np.asarray(H0, dtype=np.complex128))


def _lbfgs_accepts_every_trial(f):
    def step(ut, gt, Ft, state, lo, hi, history=8, step0=0.05, c1=1e-4, first=False):
        if not first:
            state = dict(state)
            state["F"] = -np.inf
        return f(ut, gt, Ft, state, lo, hi, history, step0, c1, first)
    return step


def _eye_like(D):
    return np.eye(D.shape[0], dtype=np.complex128)


def _with_output(fn, f):
    return lambda *a, **kw: f(fn(*a, **kw))


# ------------------------------------------------------------------ the cases
# (label, oracle attribute, variant factory taking the correct function, pins that must catch it)

CASES = [
    ("quantize: ties rounded away", "quantize", lambda f: _quantize_ties_away,
     [P.test_quantize_ties_half_even_and_clamp, P.test_quantize_matches_python_scalar_brute_force]),
    ("quantize: top level off by one", "quantize",
     lambda f: lambda u, lo, hi, L: f(u, lo, np.asarray(hi) + (np.asarray(hi) - np.asarray(lo)) / (L - 1), L + 1),
     [P.test_quantize_ties_half_even_and_clamp]),
    ("quantize: grid step (hi-lo)/L", "quantize",
     lambda f: lambda u, lo, hi, L: f(u, lo, np.asarray(lo) + (np.asarray(hi) - np.asarray(lo)) * (L - 1) / L, L),
     [P.test_quantize_grid_points_exact]),
    ("digits: most significant first", "level_digits",
     lambda f: lambda q, b, d: f(q, b, d)[..., ::-1], [P.test_digits_worked_example]),
    ("cost model: one digit too many", "plan_digits",
     lambda f: _with_output(f, lambda r: (r[0], r[1] + 1, r[2] + 1, r[3] + (r[3] // (r[2] + 1)))),
     [lambda: P.test_cost_model_printed_values("coarse_grain_example")]),
    ("table: offset on every digit", "table_thetas",
     lambda f: lambda lo, hi, L, b, d: f(lo, hi, L, b, d) + np.float64(lo),
     [P.test_table_thetas_sum_to_level_value]),
    ("level values: offset dropped", "level_values",
     lambda f: lambda q, lo, hi, L: f(q, lo, hi, L) - np.asarray(lo, dtype=np.float64),
     [P.test_table_thetas_sum_to_level_value]),
    ("Pade exponential: sign of the exponent", "expm_pade13", lambda f: lambda A: f(-A),
     [lambda: P.test_expm_pauli_closed_form(0.3)]),
    ("Pade exponential: coefficient b_3 off by 1e-6", "_B13",
     lambda f: [c * (1 + 1e-6) if j == 3 else c for j, c in enumerate(f)],
     [lambda: P.test_expm_pauli_closed_form(1.7), P.test_expm_against_scipy_and_eig]),
    ("Pade exponential: no scaling before squaring", "_THETA13", lambda f: 1e9,
     [lambda: P.test_expm_pauli_closed_form(250.0), P.test_expm_against_scipy_and_eig]),
    ("Pade exponential: transposed", "expm_pade13", lambda f: lambda A: f(A).T,
     [P.test_expm_against_scipy_and_eig]),
    ("eigen exponential: sign of t", "expm_hermitian", lambda f: lambda H, t, eig=None: f(H, -t, eig),
     [P.test_expm_against_scipy_and_eig, P.test_table_group_property_and_methods_agree]),
    ("table: drift over half a step", "build_table",
     lambda f: lambda H0, Hk, dt, lo, hi, L, b, d, method="pade": (
         f(H0, Hk, dt, lo, hi, L, b, d, method)[0], f(H0, Hk, dt / 2, lo, hi, L, b, d, method)[1]),
     [P.test_dirac_frame_step_equals_split_step, P.test_redo_error_bound_vs_quantization]),
    ("step: drift applied last", "step_propagator",
     lambda f: lambda T, D, row: D @ f(T, _eye_like(D), row),
     [P.test_dirac_frame_step_equals_split_step, P.test_redo_error_bound_vs_quantization]),
    ("step: controls in reverse order", "step_propagator",
     lambda f: lambda T, D, row: f(T[::-1], D, row[::-1]),
     [P.test_redo_error_bound_vs_quantization]),
    ("step: drift dropped", "step_propagator",
     lambda f: lambda T, D, row: f(T, _eye_like(D), row),
     [P.test_dirac_frame_step_equals_split_step, P.test_redo_error_bound_vs_quantization]),
    ("step factors: digits of the neighbouring term", "step_factors",
     lambda f: lambda T, D, row: f(T, D, np.roll(row, 1, axis=0)),
     [P.test_redo_error_bound_vs_quantization, P.test_dirac_frame_step_equals_split_step]),
    ("table: digit j scaled by b^(j-1)", "table_thetas",
     lambda f: lambda lo, hi, L, b, d: np.concatenate([f(lo, hi, L, b, d)[:1], f(lo, hi, L, b, d)[1:] / b]),
     [P.test_table_thetas_sum_to_level_value]),
    ("chain: time order reversed", "propagate", lambda f: lambda T, D, dg: f(T, D, dg[::-1]),
     [P.test_chain_time_order]),
    ("chain: last step dropped", "propagate", lambda f: lambda T, D, dg: f(T, D, dg[:-1]),
     [P.test_chain_time_order, P.test_redo_error_bound_vs_quantization]),
    ("split step: drift applied last", "split_step", lambda f: _split_step_drift_last,
     [P.test_dirac_frame_step_equals_split_step]),
    ("exact step: drift dropped", "exact_step",
     lambda f: lambda H0, Hk, dt, u: f(0.0 * np.asarray(H0), Hk, dt, u),
     [P.test_splitting_error_is_first_order, P.test_commuting_case_has_no_splitting_error]),
    ("Strang table step: Lie-Trotter instead", "strang_step_propagator",
     lambda f: lambda T, Dh, row: f(T, _eye_like(Dh), row) @ Dh @ Dh,
     [P.test_strang_table_chain_matches_split_steps_at_level_values]),
    ("half drift: a whole step", "half_drift",
     lambda f: lambda H0, dt, method="pade": f(H0, 2.0 * dt, method),
     [P.test_strang_table_chain_matches_split_steps_at_level_values]),
    ("Strang chain: time order reversed", "propagate_strang",
     lambda f: lambda T, Dh, dg: f(T, Dh, dg[::-1]),
     [P.test_strang_table_chain_matches_split_steps_at_level_values]),
    ("Strang expectation: one step late", "simulate_expectation_strang",
     lambda f: _with_output(f, lambda r: (np.concatenate([r[0][1:], r[0][-1:]]), r[1])),
     [P.test_strang_expectation_series_closed_form_and_prefix_chains]),
    ("Strang split step: whole drift on one side", "strang_split_step",
     lambda f: lambda H0, Hk, dt, u: O.split_step(H0, Hk, dt, u),
     [P.test_strang_local_error_is_third_order, P.test_strang_step_is_time_reversible]),
    ("overlap: conjugate dropped", "trace_overlap",
     lambda f: lambda UT, U: complex(np.sum(UT * U)),
     [P.test_fidelity_invariants, lambda: P.test_fidelity_closed_form_coarse_grain(1)]),
    ("fidelity: square dropped", "fidelity", lambda f: _with_output(f, np.sqrt),
     [lambda: P.test_fidelity_closed_form_coarse_grain(3)]),
    ("fidelity: normalised by N", "fidelity", lambda f: lambda UT, U: f(UT, U) * U.shape[0],
     [P.test_fidelity_invariants]),
    ("gradient: sign", "grape_gradient", lambda f: _with_output(f, lambda r: (r[0], -r[1])),
     [P.test_gradient_matches_central_differences, P.test_gradient_single_qubit_closed_form]),
    ("gradient: factor 2 dropped", "grape_gradient", lambda f: _with_output(f, lambda r: (r[0], 0.5 * r[1])),
     [P.test_gradient_matches_central_differences, P.test_gradient_single_qubit_closed_form]),
    ("gradient: steps shifted by one", "grape_gradient",
     lambda f: _with_output(f, lambda r: (r[0], np.roll(r[1], 1, axis=0))),
     [P.test_gradient_matches_central_differences]),
    ("gradient: controls swapped", "grape_gradient",
     lambda f: _with_output(f, lambda r: (r[0], r[1][:, ::-1])),
     [P.test_gradient_matches_central_differences]),
    ("state gradient: sign", "state_transfer_gradient", lambda f: _with_output(f, lambda r: (r[0], -r[1])),
     [P.test_state_transfer_gradient_matches_central_differences, P.test_state_transfer_single_qubit_closed_form]),
    ("update: no clip", "grape_update", lambda f: _grape_update_no_clip,
     [P.test_grape_update_clips_to_each_terms_grid]),
    ("update: per-pulse scale ignored", "grape_update",
     lambda f: lambda u, g, step, scale, lo, hi: f(u, g, step, None, lo, hi),
     [P.test_grape_update_one_step_closed_form]),
    ("update: another term's bounds", "grape_update",
     lambda f: lambda u, g, step, scale, lo, hi: f(u, g, step, scale, np.asarray(lo)[::-1], np.asarray(hi)[::-1]),
     [P.test_grape_update_clips_to_each_terms_grid]),
    ("step scale: comparison inverted", "grape_step_scale",
     lambda f: lambda s, F, Fp: f(s, F, Fp) if Fp is None else f(s, Fp, F),
     [P.test_grape_step_scale_schedule]),
    ("Adam ascent: no bias correction", "grape_adam_update", lambda f: _adam_no_bias_correction,
     [P.test_grape_adam_first_and_third_step_bias_correction]),
    ("Adam ascent: descends", "grape_adam_update",
     lambda f: lambda u, g, m, v, t, lr, lo, hi, **kw: f(u, -np.asarray(g), m, v, t, lr, lo, hi, **kw),
     [P.test_grape_adam_constant_gradient_steps_by_lr_and_clips, P.test_grape_ascent_reaches_a_one_qubit_target]),
    ("L-BFGS direction: sign", "lbfgs_direction", lambda f: lambda g, pairs: -f(g, pairs),
     [P.test_lbfgs_two_loop_equals_the_explicit_bfgs_matrix]),
    ("L-BFGS direction: pairs newest first", "lbfgs_direction",
     lambda f: lambda g, pairs: f(g, list(pairs)[::-1]),
     [P.test_lbfgs_two_loop_equals_the_explicit_bfgs_matrix]),
    ("L-BFGS step: every trial accepted", "grape_lbfgs_step", _lbfgs_accepts_every_trial,
     [P.test_lbfgs_backtracks_and_restarts]),
    ("polar: inverse instead of inverse root", "polar_unitary", lambda f: _polar_inverse_not_root,
     [P.test_polar_factor]),
    ("polar: Gram root on the wrong side", "polar_unitary", lambda f: _polar_wrong_side,
     [P.test_polar_factor]),
    ("expectation: one step late", "simulate_expectation",
     lambda f: _with_output(f, lambda r: (np.concatenate([r[0][1:], r[0][-1:]]), r[1])),
     [P.test_expectation_rabi_closed_form]),
    ("mixed expectation: one-sided evolution", "expect_mixed", lambda f: _expect_mixed_one_sided,
     [P.test_expect_mixed_zero_drive_closed_form, P.test_freezing_at_first_bessel_root]),
    ("GELU: tanh approximation", "gelu", lambda f: _gelu_tanh_form, [P.test_gelu_values]),
    ("GELU derivative: density term dropped", "gelu_grad", lambda f: _gelu_grad_no_density_term,
     [P.test_mlp_gradient_finite_difference]),
    ("MLP backward: weight gradient halved", "mlp_backward",
     lambda f: _with_output(f, lambda r: (r[0], [(0.5 * gw, gb) for gw, gb in r[1]])),
     [P.test_mlp_gradient_finite_difference]),
    ("MLP forward: bias ignored", "mlp_forward", lambda f: _mlp_forward_no_bias,
     [P.test_mlp_gradient_finite_difference]),
    ("MLP forward: output layer through GELU", "mlp_forward", lambda f: _mlp_forward_gelu_output,
     [P.test_mlp_gradient_finite_difference]),
    ("Adam: no bias correction", "adam_step", lambda f: _adam_step_no_bias_correction,
     [P.test_adam_first_step_is_signed_lr]),
    ("phase rotation: sign of the phase", "phase_rotation",
     lambda f: lambda phi_row, sz: f(-np.asarray(phi_row), sz),
     [P.test_phase_rotation_turns_the_x_drive_into_the_xy_drive, P.test_phase_single_spin_closed_form]),
    ("phase step: inverse rotation dropped", "phase_step_propagator",
     lambda f: lambda T, D, row, phi, sz: (
         f(T, D, row, phi, sz) @ np.linalg.inv(D) @ np.diag(O.phase_rotation(phi, sz)) @ D),
     [P.test_phase_step_at_levels_matches_the_xy_exponential, P.test_phase_single_spin_closed_form]),
    ("phase chain: time order reversed", "propagate_phase",
     lambda f: lambda T, D, dg, phi, sz: f(T, D, dg[::-1], phi[::-1], sz),
     [P.test_phase_zero_is_the_x_only_chain, P.test_phase_step_at_levels_matches_the_xy_exponential]),
    ("phase split step: inverse rotation dropped", "phase_split_step", lambda f: _phase_split_step_no_inverse,
     [P.test_phase_step_at_levels_matches_the_xy_exponential, P.test_phase_gradient_matches_central_differences]),
    ("phase gradient: phase derivative sign", "phase_gradient",
     lambda f: _with_output(f, lambda r: (r[0], r[1], -r[2])),
     [P.test_phase_gradient_matches_central_differences]),
    ("phase gradient: amplitude derivative halved", "phase_gradient",
     lambda f: _with_output(f, lambda r: (r[0], 0.5 * r[1], r[2])),
     [P.test_phase_gradient_matches_central_differences, P.test_phase_gradient_zero_phase_amplitudes_are_the_x_gradient]),
]


def _caught(pin):
    try:
        pin()
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("label,attr,variant,pins", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(label, attr, variant, pins, monkeypatch):
    monkeypatch.setattr(O, attr, variant(getattr(O, attr)))
    caught = [p for p in pins if _caught(p)]
    assert caught, f"no pin caught the planted mistake '{label}' in {attr}"


def test_every_pin_passes_on_the_oracle_as_written():
    # the catching pins are meaningful only if they pass without a planted mistake
    seen = set()
    for _, _, _, pins in CASES:
        for p in pins:
            if id(p) in seen:
                continue
            seen.add(id(p))
            p()
