"""CPU oracle for the PDFFlow hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under ``paper_2009_06635_gb300``
never imports it, and it imports nothing from there: the two implementations
share no code.  The arithmetic lives in ``pdf_oracle.c`` (plain scalar FP64
C, one point and one flavour at a time, linear-scan knot search, row-wise
Hermite in the order the paper describes); this module compiles it with gcc
and marshals numpy arrays.

Functions and the passages they follow:
  OracleGrid.xfxq2    x f(x, Q^2), Sec. 2.2 (log-bicubic, subgrids, edges) and
                      the EXTRAPOLATE box of Fig. 1 (continuation rules are a
                      reading: the paper prints none).
  OracleGrid.dxfxq2   d xf/dx, d xf/dQ^2 by forward-mode differentiation of the
                      same evaluation (no counterpart in the paper).
  OracleGrid.knot_grad  d/d(knot values) of sum_p sum_f c_pf xf_f(p), forward
                      mode seeded on each knot the evaluation read.
  OracleGrid.alphas   alpha_s(Q^2), Sec. 2.3 (log-cubic, constant extrapolation,
                      threshold subgrids).
  hermite             the cubic Hermite segment (Sec. 2.2's bicubic building block).
  rel_diff            eq. (1): |a - b| / (|b| + eps), eps = 1e-16.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pdf_oracle.c"
_LIB = _HERE / "_lib" / "libpdforacle.so"
_lib = None

EPS_EQ1 = 1e-16  # eq. (1)
UNIT_ROUNDOFF = 2.0**-53


def build(force: bool = False) -> Path:
    """Compile pdf_oracle.c with gcc (no FMA contraction, OpenMP)."""
    if not force and _LIB.exists() and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    _LIB.parent.mkdir(parents=True, exist_ok=True)
    tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(str(build()))
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.og_prepare.restype = P
    lib.og_prepare.argtypes = [i32, P, i32, P, P, i32, P, i32, P, P, ctypes.POINTER(i32)]
    lib.og_free.argtypes = [P]
    lib.og_free.restype = None
    lib.og_xfxq2.argtypes = [P, i32, P, P, P, i64, P, P, P, i32]
    lib.og_xfxq2.restype = None
    lib.og_dxfxq2.argtypes = [P, i32, i32, P, P, P, i64, P, i32]
    lib.og_dxfxq2.restype = None
    lib.og_knot_grad.argtypes = [P, P, P, i64, P, P, P]
    lib.og_knot_grad.restype = None
    lib.og_knots_read.argtypes = [P, dbl, dbl, i32, P, i32]
    lib.og_knots_read.restype = i32
    lib.og_alphas.argtypes = [P, P, i64, P, P, P, i32]
    lib.og_alphas.restype = None
    lib.og_hermite.argtypes = [dbl] * 5
    lib.og_hermite.restype = dbl
    lib.og_max_threads.argtypes = []
    lib.og_max_threads.restype = i32
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(_load().og_max_threads())


def hermite(t: float, f0: float, f1: float, m0: float, m1: float) -> float:
    return float(_load().og_hermite(t, f0, f1, m0, m1))


def rel_diff(a, b, eps: float = EPS_EQ1):
    """Relative difference of eq. (1)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / (np.abs(b) + eps)


class OracleError(ValueError):
    pass


class OracleGrid:
    """A prepared grid.  `grid` is any object with x_knots, nq, q2_knots,
    values [rows][nx][nflav], as_q2, as_vals (alpha_s may be empty)."""

    def __init__(self, grid=None, *, x_knots=None, nq=None, q2_knots=None, values=None,
                 as_q2=None, as_vals=None):
        if grid is not None:
            x_knots, nq, q2_knots, values = grid.x_knots, grid.nq, grid.q2_knots, grid.values
            as_q2, as_vals = grid.as_q2, grid.as_vals
        lib = _load()
        self._x = _f64(x_knots)
        self._nq = np.ascontiguousarray(np.asarray(nq, dtype=np.int32))
        self._q2 = _f64(q2_knots)
        self._val = _f64(values)
        self.nflav = int(self._val.shape[2])
        self._aq2 = _f64([] if as_q2 is None else as_q2)
        self._av = _f64([] if as_vals is None else as_vals)
        err = ctypes.c_int(0)
        h = lib.og_prepare(self._x.shape[0], _ptr(self._x), self._nq.shape[0], _ptr(self._nq),
                           _ptr(self._q2), self.nflav, _ptr(self._val), self._aq2.shape[0],
                           _ptr(self._aq2), _ptr(self._av), ctypes.byref(err))
        if not h:
            raise OracleError(f"oracle rejected the grid (code {err.value})")
        self._h = h
        self.nx = int(self._x.shape[0])
        self.nrows = int(self._q2.shape[0])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().og_free(h)
            self._h = None

    def _cols(self, cols):
        if cols is None:
            cols = range(self.nflav)
        return np.ascontiguousarray(np.asarray(list(cols), dtype=np.int32))

    def xfxq2(self, x, q2, cols=None, nthreads: int = 0):
        """-> (values, data_mass, marginal_flags), each [n][ncols].

        data_mass is the first-order propagation of the knot values'
        magnitudes through the same expression (sum over the knots that
        entered of |f| times the magnitudes of the coefficients on every path;
        >= |xf|, ~|xf| away from zero crossings): the scale of a relative
        error where xf crosses zero.  marginal marks
        outputs whose extrapolation branch (a positivity test) lies within
        rounding of its threshold, so another FP64 implementation may take
        the other branch."""
        x, q2 = _f64(x).ravel(), _f64(q2).ravel()
        c = self._cols(cols)
        n = x.shape[0]
        v = np.empty((n, c.shape[0]))
        m = np.empty((n, c.shape[0]))
        fl = np.zeros((n, c.shape[0]), dtype=np.uint8)
        _load().og_xfxq2(self._h, c.shape[0], _ptr(c), _ptr(x), _ptr(q2), n, _ptr(v), _ptr(m),
                         _ptr(fl), nthreads)
        return v, m, fl.astype(bool)

    def dxfxq2(self, x, q2, wrt: str, cols=None, nthreads: int = 0):
        x, q2 = _f64(x).ravel(), _f64(q2).ravel()
        c = self._cols(cols)
        d = np.empty((x.shape[0], c.shape[0]))
        _load().og_dxfxq2(self._h, {"x": 1, "q2": 2}[wrt], c.shape[0], _ptr(c), _ptr(x), _ptr(q2),
                          x.shape[0], _ptr(d), nthreads)
        return d

    def knot_grad(self, x, q2, cot, with_abs: bool = False):
        """dL/d(values) for L = sum cot * xf; with_abs also returns the sum of
        the contributions' magnitudes."""
        x, q2 = _f64(x).ravel(), _f64(q2).ravel()
        cot = _f64(cot).reshape(x.shape[0], self.nflav)
        g = np.zeros_like(self._val)
        ga = np.zeros_like(self._val) if with_abs else None
        _load().og_knot_grad(self._h, _ptr(x), _ptr(q2), x.shape[0], _ptr(cot), _ptr(g),
                             _ptr(ga) if with_abs else None)
        return (g, ga) if with_abs else g

    def knots_read(self, x: float, q2: float, col: int):
        buf = np.zeros((512, 2), dtype=np.int32)
        n = _load().og_knots_read(self._h, float(x), float(q2), int(col), _ptr(buf), 512)
        return [tuple(r) for r in buf[:n]]

    def alphas(self, q2, with_derivative: bool = False, nthreads: int = 0):
        """-> (values, data_mass) or (values, data_mass, d/dQ^2)."""
        q2 = _f64(q2).ravel()
        n = q2.shape[0]
        v, m = np.empty(n), np.empty(n)
        d = np.empty(n) if with_derivative else None
        _load().og_alphas(self._h, _ptr(q2), n, _ptr(v), _ptr(m),
                          _ptr(d) if d is not None else None, nthreads)
        return (v, m, d) if with_derivative else (v, m)
