"""The quantizer's FP32 screen, restated in numpy (CPU only).

The CUDA quantizer decides a level from an FP32 estimate
``y = fl32(fl32(fl32(v) - fl32(lo)) * fl32(1 / delta))`` wherever ``|y - rint(y)| < 1/2 - e`` with
``e = 8u|y| + 4u|lo| / |delta| + 2^-40`` (u = 2^-24), and from the FP64 subtract and divide of the
coarse-graining step (Section II) elsewhere.  The rule is exact only if the FP64 quotient
``x = fl64(fl64(v - lo) / delta)`` never lies across a half-integer from y when the screen
decides.  These tests restate the screen's arithmetic with numpy's IEEE float32 operations
and check, against the oracle's levels, on grids of every kind the library accepts:

* wherever e < 1/2 (where the screen can decide at all) the estimate's error stays within half
  of e (e is twice the first-order bound); e0 = 4u|lo|/|delta| + 2^-40 is capped at 1, which
  switches the screen off for grids offset far from zero;
* every screened decision equals the oracle's level, including values placed at distances of
  the order of e from the ties, where a bound that is too small would show.
"""
import numpy as np
import pytest

from oracle import redo_oracle as O

F32 = np.float32
U = 2.0 ** -24


def _screen(u, lo, hi, levels):
    """(decided mask, level where decided, y, e) of the FP32 screen, one term."""
    delta = (hi - lo) / (levels - 1)
    ok = 1e-30 < abs(delta) < 1e30 and abs(lo) < 1e30
    if not ok:
        n = u.shape[0]
        return np.zeros(n, bool), np.zeros(n, np.int64), np.zeros(n), np.ones(n)
    lo32 = F32(lo)
    rcp32 = F32(1.0 / delta)
    e0 = F32(min(4.0 * U * abs(lo) / abs(delta) + 2.0 ** -40, 1.0))
    with np.errstate(all="ignore"):
        # float32 roundings of v, of the subtract and of the product, as in the kernel
        y = ((u.astype(F32) - lo32).astype(F32) * rcp32).astype(F32)
        ry = np.rint(y)
        e = (np.abs(y).astype(np.float64) * 2.0 ** -21 + np.float64(e0)).astype(F32)
        decided = np.abs(y - ry) < (F32(0.5) - e)
    level = np.clip(np.nan_to_num(ry), 0, levels - 1).astype(np.int64)
    return decided, level, y.astype(np.float64), e.astype(np.float64)


GRIDS = [
    (-1.0, 1.0, 4096),
    (-2 * np.pi * 1e4, 2 * np.pi * 1e4, 4096),        # the benchmark's amplitude grid
    (0.3, 2.7, 4096),
    (-5.0, 1000.0, 65536),
    (1e3, 1e3 + 7.0, 4096),                          # far offset: the screen mostly declines
    (-3e-20, 5e-20, 4096),                           # tiny grid step
    (-1.0, 1.0, 2 ** 20),
    (-1.0, 1.0, 2 ** 24),                            # largest table: e > 1/2, every value declined
    (2.0 ** 17 * 0.25, 2.0 ** 17 * 0.25 + 1.0, 4096),  # 2^15 spans from zero: e0 capped, screen off
]


def _values(lo, hi, levels, rng):
    delta = (hi - lo) / (levels - 1)
    span = hi - lo
    uni = rng.uniform(lo - 0.2 * span, hi + 0.2 * span, size=400_000)
    # values near ties and grid points, at distances around the screen's bound
    j = rng.integers(0, levels - 1, size=4000)
    dist = np.concatenate([np.geomspace(1e-9, 0.3, 60), [0.0]])
    dist = np.concatenate([dist, -dist])
    near = []
    for c in (0.5, 0.0):
        near.append(((lo + (j + c) * delta)[:, None] + dist[None, :] * delta).ravel())
    return np.concatenate([uni] + near)


@pytest.mark.parametrize("lo,hi,levels", GRIDS)
def test_screen_error_within_half_the_bound(lo, hi, levels):
    rng = np.random.default_rng(levels % 1000 + 3)
    u = _values(lo, hi, levels, rng)
    decided, _, y, e = _screen(u, lo, hi, levels)
    delta = (hi - lo) / (levels - 1)
    x = (u - lo) / delta
    live = np.isfinite(y) & (e < 0.5)
    assert np.all(np.abs(y - x)[live] <= 0.5 * e[live])
    assert not decided[~live].any()


@pytest.mark.parametrize("lo,hi,levels", GRIDS)
def test_screened_levels_equal_the_oracle(lo, hi, levels):
    rng = np.random.default_rng(levels % 1000 + 5)
    u = _values(lo, hi, levels, rng)
    decided, level, _, _ = _screen(u, lo, hi, levels)
    q, _, _ = O.quantize(u[:, None], np.array([lo]), np.array([hi]), levels)
    assert np.array_equal(level[decided], q[decided, 0].astype(np.int64))
    if levels <= 4096 and abs(lo) * levels < 1e7 * (hi - lo):
        # on the tables the library builds the screen decides most values
        assert decided.mean() > 0.5


def test_screen_declines_non_finite_and_huge_values():
    u = np.array([np.nan, np.inf, -np.inf, 1e300, -1e300, 3.5e38, -3.5e38])
    decided, _, _, _ = _screen(u, -1.0, 1.0, 4096)
    assert not decided.any()
