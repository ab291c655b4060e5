"""Shared helpers of the GPU parity tests: tolerances and special query points.

FP64 bar (the target): |gpu - oracle| <= 1e-12 * max(|oracle|, S), with S the
oracle's data mass sum |w f| (equal to |oracle| up to a factor ~2 away from
zero crossings; it keeps the bound meaningful where xf changes sign).
Entries whose extrapolation branch the oracle flags as marginal (a positivity
test within rounding of zero) are excluded and counted.

FP32 bar: |gpu32 - oracle(x32, q2_32)| <= RTOL_FP32 * max(|oracle|, S).  The
bound follows from the arithmetic: patch coefficients rounded to FP32 (unit
roundoff 6e-8, 16 terms of size <= S), the cell position ln(x/x_i) taken in
FP32 (~1e-7 absolute, times |d xf / d ln x| <~ S), and extrapolation
amplifying relative errors by at most (1 + |p|) <~ 25 on these grids
(p the continuation parameter): 25 * ~2e-6 = 5e-5, rounded up to 1e-4.
"""
import numpy as np

RTOL_FP64 = 1e-12
RTOL_FP32 = 1e-4


def scaled_err(got, want, s):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return np.abs(got - want) / np.maximum(np.maximum(np.abs(want), s), 1e-300)


def assert_parity(got, want, s, flags, rtol, what=""):
    got = np.asarray(got, dtype=np.float64)
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), f"{what}: NaN pattern differs"
    ok = ~nan_w & ~flags
    err = scaled_err(got[ok], want[ok], s[ok])
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rtol, f"{what}: worst scaled error {worst:.3e} > {rtol:.1e}"
    return worst, int(flags.sum())


def special_points(g):
    """Knots, edges, thresholds, corners, continuation sites and invalid points."""
    xs, qs = [], []
    X, Q = np.meshgrid(g.x_knots, g.q2_knots)
    xs += list(X.ravel())
    qs += list(Q.ravel())
    x0, x1, xl = g.x_knots[0], g.x_knots[1], g.x_knots[-1]
    qmin, qmax = g.q2_knots[0], g.q2_knots[-1]
    bounds = [g.q2_knots[k] for k in np.cumsum(g.nq)[:-1]]
    xmid = [np.nextafter(x0, 0), x0, np.nextafter(x0, 2), x1, 0.5 * x0, 1e-3 * x0, 0.3, xl,
            np.nextafter(xl, 0)]
    qmid = [np.nextafter(qmin, 0), qmin, np.nextafter(qmin, np.inf), 1.01 * qmin, 0.5 * qmin, 1e-6 * qmin,
            np.nextafter(qmax, 0), qmax, np.nextafter(qmax, np.inf), 3 * qmax, 1e4 * qmax, 50.0]
    for b in bounds:
        qmid += [np.nextafter(b, 0), b, np.nextafter(b, np.inf)]
    for a in xmid:
        for b in qmid:
            xs.append(a)
            qs.append(b)
    # invalid
    xs += [0.0, -1.0, np.nan, np.inf, 0.5, 0.5, 0.5, 0.5, np.nextafter(xl, 2) if xl < 1 else 1.5]
    qs += [10.0, 10.0, 10.0, 10.0, 0.0, -5.0, np.nan, np.inf, 10.0]
    return np.array(xs, dtype=np.float64), np.array(qs, dtype=np.float64)
