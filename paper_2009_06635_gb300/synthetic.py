"""Seeded synthetic PDF grids and query sets.

This module only *produces inputs*: knot tables shaped like LHAPDF grids and
query points drawn with fixed seeds.  It holds none of the interpolation or
extrapolation arithmetic, so both the CUDA path and the CPU oracle can be fed
from it without sharing any of the method.

Knot values follow the closed form used for every synthetic set here,

    xf_i(x, Q^2) = A_i x^{a_i} (1 - x)^{b_i} (1 + c_i sqrt(x)) (1 + d_i ln(Q^2 / 2.7)),

with per-flavour parameters drawn from a numpy PCG64 stream in flavour-major
order (A, a, b, c, d for flavour 0, then flavour 1, ...), A in [0.1, 3],
a in [-0.3, 0.8], b in [2, 6], c and d in [-0.5, 0.5].  Because d < 0 is
allowed, about half the flavours change sign inside the grid, and every
flavour is exactly zero at x = 1.

The alpha_s table decreases smoothly from 0.35 to 0.09 across the Q^2 range,
one-loop-like: 1/alpha = 1/0.35 + (1/0.09 - 1/0.35) tau, tau the position of
ln Q^2 between the first and last node.

The paper's grids (NNPDF3.1 NLO, MMHT2014 NLO) are not available; these
tables stand in for them with the knot counts and ranges of typical LHAPDF
sets (Sec. 2.2 describes the grids only as LHAPDF data files).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np

# Flavour orderings (PDG ids).  21 is the gluon.
PIDS_5F = [-5, -4, -3, -2, -1, 21, 1, 2, 3, 4, 5]
PIDS_6F = [-6, -5, -4, -3, -2, -1, 21, 1, 2, 3, 4, 5, 6]

Q2_REF = 2.7  # reference scale of the d-term of the closed form


@dataclass
class Grid:
    """A PDF set in LHAPDF layout.

    x_knots : (nx,) strictly increasing, 0 < x <= 1.
    nq      : knots per Q subgrid (len = number of subgrids).
    q2_knots: (sum(nq),) concatenated; the last knot of subgrid s equals the
              first knot of subgrid s+1 (flavour threshold, duplicated).
    pids    : flavour ids, one per value column.
    values  : (sum(nq), nx, nflav) float64, the tabulated x*f(x, Q^2).
    as_q2, as_vals : alpha_s nodes (Q^2, alpha_s), non-decreasing in Q^2;
              repeated Q^2 values split alpha_s subgrids.
    """

    x_knots: np.ndarray
    nq: list
    q2_knots: np.ndarray
    pids: list
    values: np.ndarray
    as_q2: np.ndarray
    as_vals: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.x_knots.shape[0])

    @property
    def nflav(self) -> int:
        return len(self.pids)

    @property
    def nrows(self) -> int:
        return int(self.q2_knots.shape[0])


def flavour_params(nflav: int, seed: int) -> np.ndarray:
    """(nflav, 5) array of (A, a, b, c, d), drawn flavour-major from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((nflav, 5), dtype=np.float64)
    lo = [0.1, -0.3, 2.0, -0.5, -0.5]
    hi = [3.0, 0.8, 6.0, 0.5, 0.5]
    for f in range(nflav):
        for k in range(5):
            out[f, k] = rng.uniform(lo[k], hi[k])
    return out


def closed_form_values(x: np.ndarray, q2: np.ndarray, params: np.ndarray) -> np.ndarray:
    """Evaluate the closed form on the tensor grid -> (len(q2), len(x), nflav)."""
    x = np.asarray(x, dtype=np.float64)[None, :, None]
    q2 = np.asarray(q2, dtype=np.float64)[:, None, None]
    A, a, b, c, d = (params[:, k][None, None, :] for k in range(5))
    return A * x**a * (1.0 - x) ** b * (1.0 + c * np.sqrt(x)) * (1.0 + d * np.log(q2 / Q2_REF))


def alphas_nodes(q2: np.ndarray) -> np.ndarray:
    """Smoothly decreasing alpha_s values (0.35 -> 0.09) on the given Q^2 nodes."""
    lq = np.log(np.asarray(q2, dtype=np.float64))
    tau = (lq - lq[0]) / (lq[-1] - lq[0])
    return 1.0 / (1.0 / 0.35 + (1.0 / 0.09 - 1.0 / 0.35) * tau)


def geom_knots(lo: float, hi: float, n: int) -> np.ndarray:
    """n log-spaced knots with the endpoints set exactly to lo and hi."""
    k = np.geomspace(lo, hi, n)
    k[0] = lo
    k[-1] = hi
    return k


def make_grid(
    x_knots: Sequence[float],
    q2_subgrids: Sequence[Sequence[float]],
    pids: Sequence[int],
    values_fn: Callable[[np.ndarray, np.ndarray], np.ndarray] | None = None,
    params: np.ndarray | None = None,
    alphas_fn: Callable[[np.ndarray], np.ndarray] | None = None,
) -> Grid:
    """Assemble a Grid from per-subgrid Q^2 knot lists.

    values_fn(x, q2) -> (len(q2), len(x), nflav) fills the table; by default
    the closed form with `params`.  Each subgrid's first knot must equal the
    previous subgrid's last knot (the caller passes them equal).
    """
    x = np.asarray(x_knots, dtype=np.float64)
    subs = [np.asarray(s, dtype=np.float64) for s in q2_subgrids]
    q2 = np.concatenate(subs)
    nq = [int(s.shape[0]) for s in subs]
    if values_fn is None:
        assert params is not None
        vals = closed_form_values(x, q2, params)
    else:
        vals = np.asarray(values_fn(x, q2), dtype=np.float64)
    assert vals.shape == (q2.shape[0], x.shape[0], len(pids)), vals.shape
    as_vals = alphas_nodes(q2) if alphas_fn is None else np.asarray(alphas_fn(q2), dtype=np.float64)
    return Grid(
        x_knots=x,
        nq=nq,
        q2_knots=q2,
        pids=list(pids),
        values=np.ascontiguousarray(vals),
        as_q2=q2.copy(),
        as_vals=as_vals,
        params={} if params is None else {"flavour_params": params},
    )


# --------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------

def grid_single_subgrid(seed: int = 1) -> Grid:
    """One Q subgrid: 50 x knots in [1e-7, 1], 40 Q^2 knots in [2.7, 1e8], 11 flavours."""
    params = flavour_params(len(PIDS_5F), seed)
    return make_grid(geom_knots(1e-7, 1.0, 50), [geom_knots(2.7, 1e8, 40)], PIDS_5F, params=params)


# Three Q subgrids split at the charm and bottom thresholds Q = 1.51 and
# 4.92 GeV, lowest knot Q = 1.0 GeV, highest 1e5 GeV (12 + 15 + 25 knots,
# boundary knots duplicated -> 52 rows); 196 x knots in [1e-9, 1]; 13 flavours.
Q_THRESHOLDS = (1.51, 4.92)
Q_RANGE = (1.0, 1e5)
SUBGRID_KNOTS = (12, 15, 25)


def grid_full(seed: int = 1) -> Grid:
    params = flavour_params(len(PIDS_6F), seed)
    qb = [Q_RANGE[0], Q_THRESHOLDS[0], Q_THRESHOLDS[1], Q_RANGE[1]]
    q2b = [q * q for q in qb]
    subs = [geom_knots(q2b[s], q2b[s + 1], SUBGRID_KNOTS[s]) for s in range(3)]
    return make_grid(geom_knots(1e-9, 1.0, 196), subs, PIDS_6F, params=params)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def queries_single_subgrid(n: int = 10_000, seed: int = 2):
    """In-grid queries for grid_single_subgrid: ln x ~ U[ln 1e-7, 0], ln Q^2 ~ U[ln 2.7, ln 1e8]."""
    r = _rng(seed)
    lx = r.uniform(np.log(1e-7), 0.0, n)
    lq2 = r.uniform(np.log(2.7), np.log(1e8), n)
    return np.exp(lx), np.exp(lq2)


def queries_full(n: int = 10_000_000, seed: int = 3):
    """Queries for grid_full: ln x ~ U[ln 1e-10, 0], ln Q ~ U[0, ln 2e5] (some fall outside the grid)."""
    r = _rng(seed)
    lx = r.uniform(np.log(1e-10), 0.0, n)
    lqq = r.uniform(0.0, np.log(2e5), n)
    return np.exp(lx), np.exp(2.0 * lqq)


QUERY_CLASSES = ("in", "lowx", "highq", "lowq", "lowx_highq", "lowx_lowq")


def queries_class(grid: Grid, cls: str, n: int, seed: int = 3):
    """n queries of one class of point (for profiling one class at a time):
    drawn from the queries_full law widened to Q in [0.1, 2e5] GeV, keeping
    those whose x lies below, inside or above the grid's x range and Q^2
    below, inside or above its Q^2 range as `cls` names ("in", "lowx",
    "highq", "lowq", "lowx_highq", "lowx_lowq")."""
    want_lowx = cls.startswith("lowx")
    want_q = "highq" if cls.endswith("highq") else "lowq" if cls.endswith("lowq") else "in"
    r = _rng(seed)
    xs, qs, have = [], [], 0
    while have < n:
        m = max(4 * (n - have), 1024)
        x = np.exp(r.uniform(np.log(1e-10), 0.0, m))
        q2 = np.exp(2.0 * r.uniform(np.log(0.1), np.log(2e5), m))
        lowx = x < grid.x_knots[0]
        qcls = np.where(q2 > grid.q2_knots[-1], "highq", np.where(q2 < grid.q2_knots[0], "lowq", "in"))
        keep = (lowx == want_lowx) & (qcls == want_q)
        xs.append(x[keep])
        qs.append(q2[keep])
        have += int(keep.sum())
    return np.concatenate(xs)[:n], np.concatenate(qs)[:n]


SQRT_S = 13000.0  # GeV


def events_mc(n: int = 1_000_000, seed: int = 4):
    """Monte Carlo event batch: ln x1, ln x2 ~ U[ln 1e-6, 0]; Q^2 = x1 x2 s is formed by the kernel."""
    r = _rng(seed)
    lx1 = r.uniform(np.log(1e-6), 0.0, n)
    lx2 = r.uniform(np.log(1e-6), 0.0, n)
    return np.exp(lx1), np.exp(lx2), SQRT_S * SQRT_S


def adjoint_inputs(n: int = 1_000_000, nflav: int = 13, seed_pts: int = 5, seed_cot: int = 6):
    """Points from the queries_full law and standard-normal cotangents (n, nflav)."""
    x, q2 = queries_full(n, seed_pts)
    cot = _rng(seed_cot).standard_normal((n, nflav))
    return x, q2, cot


def ingrid_samples(grid: Grid, n: int, seed: int):
    """Log-uniform (x, Q^2) strictly inside the grid's range."""
    r = _rng(seed)
    lx = r.uniform(np.log(grid.x_knots[0]), np.log(grid.x_knots[-1]), n)
    lq2 = r.uniform(np.log(grid.q2_knots[0]), np.log(grid.q2_knots[-1]), n)
    return np.exp(lx), np.exp(lq2)


# --------------------------------------------------------------------------
# Learned surrogate: seeded initial parameters (random numbers the training
# draws, passed to the GPU and to any checker alike)
# --------------------------------------------------------------------------

SURROGATE_WIDTH = 128
SURROGATE_NFREQ = 16


def surrogate_init(nflav: int, seed: int = 9, freq_sigma: float = 2.0):
    """-> (params float32 flat, freq float32 [16][2]).

    params: W1 [128][32], b1 [128], W2..W4 [128][128], b2..b4, W5 [nflav][128],
    b5 [nflav]; weights uniform in +-sqrt(6/fan_in) (He-uniform), biases zero.
    freq: the fixed Fourier-feature frequencies, normal with sigma freq_sigma."""
    r = _rng(seed)
    W = SURROGATE_WIDTH
    shapes = [(W, 2 * SURROGATE_NFREQ), (W, W), (W, W), (W, W), (nflav, W)]
    parts = []
    for (o, i) in shapes:
        lim = np.sqrt(6.0 / i)
        parts.append(r.uniform(-lim, lim, o * i))
        parts.append(np.zeros(o))
    params = np.concatenate(parts).astype(np.float32)
    freq = r.normal(0.0, freq_sigma, (SURROGATE_NFREQ, 2)).astype(np.float32)
    return params, freq


# --------------------------------------------------------------------------
# Members (replicas) of the three-subgrid set, and the fitting x grid
# --------------------------------------------------------------------------

def grid_members(nmem: int, seed: int = 12, base_seed: int = 1, spread: float = 0.05):
    """-> (Grid with member 0's values, values [nmem][rows][nx][nflav]).

    Member m perturbs the base flavour parameters with seeded normals:
    A *= 1 + spread N, a += 0.2 spread N, b, c, d += spread N (drawn member by
    member, parameter-major within a member)."""
    g = grid_full(base_seed)
    base = g.params["flavour_params"]
    nf = base.shape[0]
    r = _rng(seed)
    vals = np.empty((nmem,) + g.values.shape)
    for m in range(nmem):
        p = base.copy()
        p[:, 0] *= 1.0 + spread * r.standard_normal(nf)
        p[:, 1] += 0.2 * spread * r.standard_normal(nf)
        p[:, 2] += spread * r.standard_normal(nf)
        p[:, 3] += spread * r.standard_normal(nf)
        p[:, 4] += spread * r.standard_normal(nf)
        vals[m] = closed_form_values(g.x_knots, g.q2_knots, p)
    g0 = make_grid(g.x_knots, [g.q2_knots[a:a + n] for a, n in zip(np.cumsum([0] + g.nq)[:-1], g.nq)], g.pids,
                   values_fn=lambda x, q: vals[0])
    return g0, vals


FIT_Q = 1.65  # GeV, the parametrisation scale of an NNPDF3.1-style fit


def fit_points(n: int = 2415, q: float = FIT_Q):
    """x grid of a fit's convolution tables: n points log-spaced in [1e-9, 1), at Q^2 = q^2."""
    x = np.geomspace(1e-9, 1.0, n + 1)[:-1]
    return x, np.full(n, q * q)


# --------------------------------------------------------------------------
# LHAPDF6 text files (lhagrid1) of a synthetic set
# --------------------------------------------------------------------------

def write_lhapdf(grid: Grid, set_dir, member_values=None, digits: int = 17):
    """Write grid as an LHAPDF6 set directory (NAME.info + NAME_%04d.dat, one
    file per member; member_values [nmem][rows][nx][nflav] or the grid's own
    values).  Q knots are written as sqrt(Q^2); with 17 digits every number
    reads back exactly (the Q^2 knots as sqrt(Q^2)^2).  Returns the paths."""
    import os
    d = os.fspath(set_dir).rstrip("/")
    name = os.path.basename(d)
    os.makedirs(d, exist_ok=True)
    fmt = f"%.{digits - 1}e"
    members = [grid.values] if member_values is None else list(member_values)
    nums = lambda a: " ".join(fmt % v for v in np.asarray(a, dtype=np.float64).ravel())  # noqa: E731
    with open(os.path.join(d, name + ".info"), "w") as f:
        f.write(f"SetDesc: \"synthetic LHAPDF-shaped set written by write_lhapdf\"\n")
        f.write("Format: lhagrid1\n")
        f.write(f"NumMembers: {len(members)}\n")
        f.write("Flavors: [" + ", ".join(str(p) for p in grid.pids) + "]\n")
        f.write(f"XMin: {fmt % grid.x_knots[0]}\nXMax: {fmt % grid.x_knots[-1]}\n")
        if len(grid.as_q2):
            qs = [fmt % q for q in np.sqrt(np.asarray(grid.as_q2))]
            f.write("AlphaS_Type: ipol\n")
            # a list continued over lines, as long metadata lists often are
            f.write("AlphaS_Qs: [" + ",\n  ".join(", ".join(qs[i:i + 8]) for i in range(0, len(qs), 8)) + "]\n")
            f.write("AlphaS_Vals: [" + ", ".join(fmt % v for v in grid.as_vals) + "]\n")
    paths = []
    starts = np.concatenate([[0], np.cumsum(grid.nq)])
    for m, vals in enumerate(members):
        p = os.path.join(d, f"{name}_{m:04d}.dat")
        with open(p, "w") as f:
            f.write(f"PdfType: {'central' if m == 0 else 'replica'}\nFormat: lhagrid1\n---\n")
            for s in range(len(grid.nq)):
                r0, r1 = starts[s], starts[s + 1]
                f.write(nums(grid.x_knots) + "\n")
                f.write(nums(np.sqrt(grid.q2_knots[r0:r1])) + "\n")
                f.write(" ".join(str(p_) for p_ in grid.pids) + "\n")
                block = np.asarray(vals)[r0:r1]  # [nq][nx][nf]
                for ix in range(len(grid.x_knots)):
                    for iq in range(r1 - r0):
                        f.write(nums(block[iq, ix]) + "\n")
                f.write("---\n")
        paths.append(p)
    return paths

