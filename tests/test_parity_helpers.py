"""The parity checks themselves (tests/parity.py, tests/surrogate_bounds.py)
on the CPU: outputs within their bounds pass, and one element moved by ten
times its bound fails, for the FP64 bar, the FP32 per-class bound and the
surrogate's element-wise check."""
import numpy as np
import pytest

import parity
import surrogate_bounds as sb


@pytest.fixture(scope="module")
def case(synth, oracle_mod):
    g = synth.grid_full()
    og = oracle_mod.OracleGrid(g)
    x, q2 = synth.queries_full(3000, 77)
    sx, sq = parity.special_points(g)
    x, q2 = np.concatenate([x, sx]), np.concatenate([q2, sq])
    v, s, fl = og.xfxq2(x, q2)
    return g, x, q2, v, s, fl


def _inside(want, s, tol, rng):
    """Outputs moved by a random fraction (up to half) of their bound."""
    scale = np.maximum(np.abs(want), s) * tol
    return want + rng.uniform(-0.5, 0.5, want.shape) * np.nan_to_num(scale)


def _one_out(got, want, s, tol, k):
    bad = got.copy()
    flat = bad.reshape(-1)
    scale = np.maximum(np.abs(want), s).reshape(-1) * np.broadcast_to(tol, want.shape).reshape(-1)
    flat[k] = want.reshape(-1)[k] + 10.0 * scale[k]
    return bad


def test_fp64_bar_passes_inside_and_fails_at_ten_times(case):
    g, x, q2, v, s, fl = case
    rng = np.random.default_rng(1)
    got = _inside(v, s, parity.RTOL_FP64, rng)
    parity.assert_parity(got, v, s, fl, parity.RTOL_FP64, "inside")
    ok = np.flatnonzero((~np.isnan(v) & ~fl).reshape(-1))
    for k in rng.choice(ok, 5, replace=False):
        with pytest.raises(AssertionError):
            parity.assert_parity(_one_out(got, v, s, parity.RTOL_FP64, k), v, s, fl, parity.RTOL_FP64, "moved")


def test_fp32_bound_passes_inside_and_fails_at_ten_times(case):
    g, x, q2, v, s, fl = case
    rng = np.random.default_rng(2)
    tol = parity.fp32_bound(g, x, q2)[:, None]
    got = _inside(v, s, tol, rng)
    parity.assert_fp32(g, x, q2, got, v, s, fl, "inside")
    ok = ~np.isnan(v) & ~fl
    cls = parity.point_classes(g, x, q2)
    # one element of each class present, in-grid points first
    for c in range(6):
        rows = np.flatnonzero((cls == c) & ok.all(axis=1))
        if rows.size == 0:
            continue
        k = int(rows[0]) * v.shape[1] + int(rng.integers(v.shape[1]))
        with pytest.raises(AssertionError):
            parity.assert_fp32(g, x, q2, _one_out(got, v, s, tol, k), v, s, fl, f"class {c} moved")


def test_fp32_bound_is_near_the_measured_error():
    """The in-grid FP32 bound (20u) sits within a few times the worst error
    the FP32 path has shown in-grid (6.2u), not hundreds of times above it."""
    assert parity.FP32_IN * parity.U32 < 4.0 * 6.2 * parity.U32


def test_surrogate_check_fails_at_ten_times_its_bound():
    rng = np.random.default_rng(3)
    want = rng.normal(size=(50, 13))
    bound = np.abs(rng.normal(size=want.shape)) * 1e-3 + 1e-6
    got = want + rng.uniform(-0.9, 0.9, want.shape) * bound
    sb.assert_within(got, want, bound, "inside")
    for k in rng.choice(want.size, 5, replace=False):
        bad = got.copy().reshape(-1)
        bad[k] = want.reshape(-1)[k] + 10.0 * bound.reshape(-1)[k]
        with pytest.raises(AssertionError):
            sb.assert_within(bad.reshape(want.shape), want, bound, "moved")
