"""Shared helpers of the GPU parity tests: tolerances and special query points.

FP64 bar (the target): |gpu - oracle| <= 1e-12 * max(|oracle|, S), with S the
oracle's data mass: the knot values' magnitudes propagated to first order
through the same expression (>= |oracle|; near it away from zero crossings,
(1 + 2|p|) times it through a log-linear continuation with parameter p;
pinned in test_oracle_mass_pins).  It keeps the bound meaningful where xf
changes sign.  Entries whose extrapolation branch the oracle flags as
marginal (a positivity test within rounding of zero) are excluded and
counted.  eq1_report states the paper's own eq. (1) beside it.

FP32 bar, per point class (fp32_bound), in units of u = 2^-24 of S, against
the oracle at the float inputs.  An in-grid item is the cell's control
points rounded to float (1u of S: the Bernstein weights are non-negative and
sum to one, and sum B|b| <= S), times Bernstein weights built from the
position with three roundings each (3u per direction: 6u), contracted as four
4-term FMA rows, a product and a pairwise sum (7u), at a position t taken
relative to the nearer knot with ~6 roundings (6u of t, times |t dxf/dt| <~ S:
6u): 20u = 1.2e-6.  A continuation rule acts on site values whose errors the
mass already carries ((1 + 2|p|) S for the pair rule, so a relative error of
the sites stays a relative error of S); what it adds is its own arithmetic:
logf, expf, the quotient and product (~1 ulp each) and the parameter p taken
in float (|p ln r| 3u of v, and |p| <= (1 + 2|p|) / 2): +6u per rule.  The
low-Q^2 rule also rounds the exponent (gamma rho + 1 - rho) ln rho, whose
error 3u |ln rho| is relative to v and not covered by S (for rho -> 0,
S -> |v|): +3u |ln rho|.
"""
import numpy as np

RTOL_FP64 = 1e-12
U32 = 2.0**-24
FP32_IN, FP32_RULE, FP32_LOWQ_LOG = 20.0, 6.0, 3.0  # units of U32, see above
EPS_EQ1 = 1e-16  # eq. (1)


def scaled_err(got, want, s):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return np.abs(got - want) / np.maximum(np.maximum(np.abs(want), s), 1e-300)


def assert_parity(got, want, s, flags, rtol, what=""):
    """rtol: a scalar, or one bound per point (broadcast over the columns)."""
    got = np.asarray(got, dtype=np.float64)
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), f"{what}: NaN pattern differs"
    ok = ~nan_w & ~flags
    tol = np.broadcast_to(np.asarray(rtol, dtype=np.float64).reshape(-1, *([1] * (want.ndim - 1)))
                          if np.ndim(rtol) else rtol, want.shape)
    err = scaled_err(got[ok], want[ok], s[ok])
    ratio = err / tol[ok]
    worst = float(err.max()) if err.size else 0.0
    if ratio.size and ratio.max() > 1.0:
        k = int(np.argmax(ratio))
        raise AssertionError(f"{what}: scaled error {err[k]:.3e} > its bound {tol[ok][k]:.3e} "
                             f"(worst scaled error {worst:.3e})")
    return worst, int(flags.sum())


def point_classes(g, x, q2):
    """0 in-grid, 1 x below, 2 Q^2 above, 3 Q^2 below, 4 x below and Q^2
    above, 5 x below and Q^2 below, 6 invalid (host bookkeeping)."""
    x, q2 = np.asarray(x, dtype=np.float64), np.asarray(q2, dtype=np.float64)
    valid = (x > 0) & (x <= g.x_knots[-1]) & (q2 > 0) & np.isfinite(q2)
    lowx = x < g.x_knots[0]
    lowq, highq = q2 < g.q2_knots[0], q2 > g.q2_knots[-1]
    cls = np.where(lowx, np.where(highq, 4, np.where(lowq, 5, 1)), np.where(highq, 2, np.where(lowq, 3, 0)))
    return np.where(valid, cls, 6)


def fp32_bound(g, x, q2):
    """Per-point FP32 bound (scaled error) of the class each float input falls in."""
    cls = point_classes(g, x, q2)
    rules = np.choose(np.minimum(cls, 6), [0, 1, 1, 1, 2, 2, 0])
    with np.errstate(divide="ignore", invalid="ignore"):
        lr = np.abs(np.log(np.asarray(q2, dtype=np.float64) / g.q2_knots[0]))
    lowq = (cls == 3) | (cls == 5)
    units = FP32_IN + FP32_RULE * rules + FP32_LOWQ_LOG * np.where(lowq, lr, 0.0)
    return units * U32


FP32_ALPHAS = 10.0  # units of U32: three FMA steps, the rounded cubic (1u), the position (~4u of u, times
                   # |d alpha / du| / alpha << 1) and the constant ends (exact)
CLASS_NAMES = ("in", "lowx", "highq", "lowq", "lowx_highq", "lowx_lowq", "invalid")


def assert_fp32(g, x, q2, got, want, s, flags, what=""):
    """FP32 outputs against the oracle at the float inputs x, q2 (float64
    copies of the floats), each point held to its class's bound.  Returns
    the worst scaled error per column and per class (in units of u)."""
    bound = fp32_bound(g, x, q2)
    assert_parity(got, want, s, flags, bound, what)
    ok = ~np.isnan(want) & ~flags
    err = np.where(ok, scaled_err(got, want, s), 0.0)
    cls = point_classes(g, x, q2)
    per_class = {CLASS_NAMES[c]: float(err[cls == c].max() / U32) for c in range(6) if (cls == c).any()}
    return err.max(axis=0), per_class


def eq1_report(got, want, s, flags, cancel=1e-3):
    """The paper's eq. (1), |got - want| / (|want| + 1e-16), per column: its
    maximum over the outputs that are not at a zero crossing of xf
    (|want| >= cancel * S: no cancellation by more than 1/cancel), and how
    many outputs were left out as crossing zero."""
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    ok = ~np.isnan(want) & ~flags
    far = ok & (np.abs(want) >= cancel * s)
    r = np.abs(got - want) / (np.abs(want) + EPS_EQ1)
    per = np.where(far, r, 0.0).max(axis=0) if want.ndim > 1 else np.array([np.where(far, r, 0.0).max()])
    return {"eq1_max_per_column": [float(v) for v in per], "eq1_max": float(per.max()),
            "near_zero_excluded": int((ok & ~far).sum()), "outputs": int(ok.sum()),
            "near_zero": f"|oracle| < {cancel:g} x data mass"}


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
