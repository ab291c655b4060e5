"""The FP64 evaluation kernels' own elementary functions (tang.cuh: Tang's
table-driven logarithm and exponential, and the Newton division; ffmath.cuh:
their float-float counterparts used by the continuation rules) against the C
library's, which round within one ulp: over the ranges the kernels use, and
at the special values they must get right."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2009_06635_gb300")


@pytest.fixture(scope="module")
def grid(synth):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return P.pdf_load_grid(synth.grid_single_subgrid())


def run(G, fn, a, b=None):
    from paper_2009_06635_gb300 import _native
    ad = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    bd = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64)).cuda() if b is not None else None
    out = torch.empty_like(ad)
    _native.check_probe(_native.load_probe().pdf_probe_math(G.handle, fn, ctypes.c_void_p(ad.data_ptr()),
                                                ctypes.c_void_p(bd.data_ptr() if bd is not None else 0), len(a),
                                                ctypes.c_void_p(out.data_ptr()), None), "pdf_probe_math")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def test_log(grid):
    r = np.random.default_rng(1)
    a = np.concatenate([np.exp(r.uniform(-700, 700, 200_000)), r.uniform(0.5, 2.0, 200_000),
                        1 + r.uniform(-1e-3, 1e-3, 100_000), [1.0, 2.0, 0.5, np.nextafter(1, 0), np.nextafter(1, 2),
                                                              5e-324, 1e-310, np.finfo(float).max]])
    got = run(grid, 0, a)
    want = np.log(a)
    # the documented bound: two roundings (e ln2 + ln F, then + log1p(u)),
    # the rounding of ln2 times the exponent, and the degree-5 series'
    # truncation (|u|^6 / 6 <= 2^-54 / 6): 2 ulp of ln a or 2e-17 absolute
    err = np.abs(got - want)
    assert np.all(err <= 2 * np.spacing(np.abs(want)) + 2e-17), (err / (2 * np.spacing(np.abs(want)) + 2e-17)).max()
    # near a = 1 the result is not the difference of two rounded logarithms
    # (a just below 1 reads ln(F/2) from its table): no cancellation beyond that bound
    near = np.abs(want) < 1e-4
    assert np.all(err[near] <= 2 * np.spacing(np.abs(want[near]))), (err[near] / np.spacing(np.abs(want[near]))).max()
    assert got[-8] == 0.0 and got[-7] == np.log(2.0)
    assert np.array_equal(run(grid, 0, np.array([0.0, np.inf])), np.array([-np.inf, np.inf]))
    assert np.isnan(run(grid, 0, np.array([np.nan]))[0])


def test_exp(grid):
    r = np.random.default_rng(2)
    y = np.concatenate([r.uniform(-699, 699, 300_000), r.uniform(-1e-3, 1e-3, 100_000), [0.0, -0.0, 1e-300,
                                                                                           -745.2, 709.9, 800.0]])
    got = run(grid, 1, y)
    with np.errstate(over="ignore"):
        want = np.exp(y)
    fin = np.isfinite(want) & (want > 1e-300)
    assert np.all(ulps(got[fin], want[fin]) <= 2.0), ulps(got[fin], want[fin]).max()
    assert got[-6] == 1.0 and got[-5] == 1.0 and np.isinf(got[-1])


def test_division(grid):
    r = np.random.default_rng(3)
    a = r.normal(0, 1, 300_000) * 10.0 ** r.integers(-30, 30, 300_000)
    b = r.normal(0, 1, 300_000) * 10.0 ** r.integers(-30, 30, 300_000)
    got = run(grid, 2, a, b)
    want = a / b
    assert np.all(ulps(got, want) <= 2.0), ulps(got, want).max()
    special = run(grid, 2, np.array([1.0, 1.0, 1.0, 0.0]), np.array([0.0, 5e-324, np.inf, 2.0]))
    assert np.isinf(special[0]) and special[1] == 1.0 / 5e-324 and special[2] == 0.0 and special[3] == 0.0


def test_float_float_log(grid):
    """ln r of the continuation rules (r a quotient of site values, which the
    rules keep in [2^-100, 2^100], where the low part of a float pair is a
    normal float): absolute error within 2e-14 + 2e-14 |ln r| (the table's and
    the series' float-float roundings, ~2^-47, and three float-float additions
    of terms as large as |ln r|, each within ~2^-48 of its result)."""
    r = np.random.default_rng(4)
    a = np.concatenate([np.exp(r.uniform(-69, 69, 200_000)), r.uniform(0.3, 3.0, 200_000),
                        1 + r.uniform(-1e-4, 1e-4, 100_000), [1.0, 2.0, 0.5, 1.0 + 2.0**-30, 1.0 - 2.0**-30]])
    a = a.astype(np.float32).astype(np.float64) * (1 + r.uniform(-2.0**-30, 2.0**-30, a.size))  # use the low part
    got = run(grid, 3, a)
    want = np.log(a)
    err = np.abs(got - want)
    bound = 2e-14 + 2e-14 * np.abs(want)
    assert np.all(err <= bound), (err / bound).max()


def test_float_float_exp(grid):
    """e^y for the exponents the rules send here (|y| < 64: the result's low
    part stays a normal float): relative error within (1 + |y|) 1e-14."""
    r = np.random.default_rng(5)
    y = np.concatenate([r.uniform(-63.9, 63.9, 300_000), r.uniform(-1e-3, 1e-3, 100_000), [0.0, 1e-20, -1e-20, 50.0]])
    got = run(grid, 4, y)
    want = np.exp(y)
    rel = np.abs(got - want) / want
    bound = (1 + np.abs(y)) * 1e-14
    assert np.all(rel <= bound), (rel / bound).max()
    assert got[-4] == 1.0


def test_float_float_division(grid):
    r = np.random.default_rng(6)
    a = r.normal(0, 1, 300_000) * 10.0 ** r.integers(-15, 15, 300_000)
    b = r.normal(0, 1, 300_000) * 10.0 ** r.integers(-15, 15, 300_000)
    got = run(grid, 5, a, b)
    want = a / b
    rel = np.abs(got - want) / np.abs(want)
    assert np.all(rel <= 4e-14), rel.max()


def test_float_float_cell_positions(synth):
    """The evaluation kernels' in-grid positions t = ln(x/x_i) / ln(x_(i+1)/x_i)
    and 1 - t, taken in float-float from the bit patterns (ffpos.cuh), against
    40-digit decimal logarithms: within 5e-14 absolute everywhere (the FP64
    path's own rounding is ~2e-14), exactly 0 and 1 on the knots, and within
    1e-13 relative for the small 1 - t next to x = 1, where the data vanish."""
    from decimal import Decimal, getcontext

    getcontext().prec = 40
    g = synth.grid_full()
    G = P.pdf_load_grid(g)
    xk = g.x_knots
    r = np.random.default_rng(8)
    i = r.integers(0, len(xk) - 1, 3000)
    x = np.exp(r.uniform(np.log(xk[i]), np.log(xk[i + 1])))
    near = np.concatenate([xk[1:-1, None] * (1 + 10.0 ** -np.arange(1, 14))[None, :],
                           xk[2:, None] * (1 - 10.0 ** -np.arange(1, 14))[None, :]]).ravel()[::7]
    top = 1.0 - 10.0 ** -np.arange(1, 14)
    x = np.concatenate([x, near, top, xk])
    t, ts = run(G, 6, x), run(G, 7, x)
    cell = np.searchsorted(xk, x, side="right") - 1
    for k in range(x.size):
        c = cell[k]
        if c == len(xk) - 1:  # the last knot itself
            assert t[k] == 0.0 and ts[k] == 1.0
            continue
        lo, hi = Decimal(float(xk[c])).ln(), Decimal(float(xk[c + 1])).ln()
        et = (Decimal(float(x[k])).ln() - lo) / (hi - lo)
        assert abs(Decimal(float(t[k])) - et) <= Decimal("5e-14"), (x[k], float(t[k]), float(et))
        assert abs(Decimal(float(ts[k])) - (1 - et)) <= Decimal("5e-14"), (x[k], float(ts[k]), float(1 - et))
        if x[k] == xk[c]:
            assert t[k] == 0.0 and ts[k] == 1.0
    for k in range(x.size - len(xk) - len(top), x.size - len(xk)):  # next to x = 1
        ets = 1 - (Decimal(float(x[k])).ln() - Decimal(float(xk[-2])).ln()) / (-Decimal(float(xk[-2])).ln())
        assert abs(Decimal(float(ts[k])) - ets) <= Decimal("1e-13") * ets, (x[k], float(ts[k]), float(ets))


def test_integer_split_to_float_pairs(grid):
    """The adjoint's split of a double into a float pair without FP64
    conversions (ffsplit.cuh): hi is the double's top 24 significant bits
    (truncated, so |hi| <= |a|), hi + lo is a to within 2^-48 |a| with lo of
    a's sign, zeros split to zeros, and values outside 2^+-50 are refused."""
    r = np.random.default_rng(11)
    mag = np.exp2(r.uniform(-50, 50, 200_000))
    a = np.concatenate([mag * r.choice([-1.0, 1.0], mag.size), [0.0, -0.0, 1.0, -1.0, 2.0 ** -50,
                        np.nextafter(2.0 ** 50, 0), 1 + 2.0 ** -52, 1 - 2.0 ** -53, 3.0 ** 30]])
    hi = run(grid, 9, a)
    top = (a.view(np.int64) & ~np.int64((1 << 29) - 1)).view(np.float64)  # the top 24 significant bits
    assert np.array_equal(hi, top)
    both = run(grid, 8, a)
    assert (np.abs(both - a) <= 2.0 ** -48 * np.abs(a)).all()
    assert (np.abs(both) >= np.abs(hi)).all()  # lo has a's sign
    assert np.array_equal(run(grid, 8, np.array([0.0])), [0.0])
    out = run(grid, 8, np.array([2.0 ** 50, 2.0 ** -51, -2.0 ** 60, np.inf, np.nan]))
    assert np.isnan(out).all()
