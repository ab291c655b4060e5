"""PyTorch-facing API over the C ABI (names as in include/pdf_gb300.h).

    grid = pdf_load_grid(synthetic.grid_full())      # PDFFlow mkPDF (Sec. 2.1)
    out  = xfxq2_all_flavours(grid, x, q2)           # xfxQ2_allpid
    a    = alphas_q2(grid, q2)                       # alphas_Q2
    a    = alphas_q(grid, q)                         # alphas_Q (Q in GeV)

Tensors must be CUDA, contiguous, float64 (or float32 for the *_f32 paths);
work is enqueued on torch's current stream of the tensors' device.  PyTorch
only provides device memory and the stream; the evaluation is the library's.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import PdfError, check


def _stream_handle(dev: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _dev_ptr(t: torch.Tensor, dtype, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """A loaded PDF set (owns the device-side handle)."""

    def __init__(self, handle: int, pids, device: torch.device, nx: int, nrows: int, nmem: int = 1):
        self._h = ctypes.c_void_p(handle)
        self.pids = list(pids)
        self.nflav = len(self.pids)
        self.nx = nx
        self.nrows = nrows
        self.nmem = nmem
        self.device = device

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise PdfError(-1, "grid has been freed")
        return self._h

    def free(self):
        if self._h:
            check(_native.load().pdf_free_grid(self._h), "pdf_free_grid")
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def column(self, pid: int) -> int:
        return int(_native.load().pdf_grid_pid_column(self.handle, int(pid)))

    def invalid_count(self) -> int:
        c = ctypes.c_ulonglong(0)
        check(_native.load().pdf_grid_invalid_count(self.handle, ctypes.byref(c)), "pdf_grid_invalid_count")
        return int(c.value)

    def reset_invalid_count(self):
        check(_native.load().pdf_grid_reset_invalid_count(self.handle), "pdf_grid_reset_invalid_count")


def pdf_load_grid(grid=None, *, x_knots=None, nq=None, q2_knots=None, pids=None, values=None,
                  as_q2=None, as_vals=None, device=None, member_values=None) -> Grid:
    """Load a PDF set (any object with x_knots, nq, q2_knots, pids, values,
    as_q2, as_vals, or the same as keywords) onto the current CUDA device.
    member_values [nmem][rows][nx][nflav] loads a member set sharing the knots."""
    if grid is not None:
        x_knots, nq, q2_knots, pids, values = grid.x_knots, grid.nq, grid.q2_knots, grid.pids, grid.values
        as_q2, as_vals = grid.as_q2, grid.as_vals
    lib = _native.load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    xk = np.ascontiguousarray(x_knots, dtype=np.float64)
    nqa = np.ascontiguousarray(nq, dtype=np.int32)
    q2k = np.ascontiguousarray(q2_knots, dtype=np.float64)
    pa = np.ascontiguousarray(pids, dtype=np.int32)
    va = np.ascontiguousarray(values, dtype=np.float64)
    aq = np.ascontiguousarray([] if as_q2 is None else as_q2, dtype=np.float64)
    av = np.ascontiguousarray([] if as_vals is None else as_vals, dtype=np.float64)
    if va.ndim != 3 or va.shape != (q2k.shape[0], xk.shape[0], pa.shape[0]):
        raise PdfError(-2, f"values shape {va.shape} != (rows, nx, nflav)")
    mv = None
    if member_values is not None:
        mv = np.ascontiguousarray(member_values, dtype=np.float64)
        if mv.ndim != 4 or mv.shape[1:] != va.shape:
            raise PdfError(-2, f"member_values shape {mv.shape} != (nmem, rows, nx, nflav)")
    d = _native.GridDesc(
        int(xk.shape[0]), xk.ctypes.data, int(nqa.shape[0]), nqa.ctypes.data, q2k.ctypes.data,
        int(pa.shape[0]), pa.ctypes.data, va.ctypes.data, int(aq.shape[0]),
        aq.ctypes.data if aq.size else None, av.ctypes.data if av.size else None)
    h = ctypes.c_void_p(None)
    with torch.cuda.device(dev):
        if mv is None:
            check(lib.pdf_load_grid(ctypes.byref(d), ctypes.byref(h)), "pdf_load_grid")
        else:
            check(lib.pdf_load_grid_members(ctypes.byref(d), int(mv.shape[0]), mv.ctypes.data, ctypes.byref(h)),
                  "pdf_load_grid_members")
    return Grid(h.value, pa.tolist(), dev, int(xk.shape[0]), int(q2k.shape[0]), 1 if mv is None else int(mv.shape[0]))


def _out(out, shape, like: torch.Tensor):
    if out is None:
        return torch.empty(shape, dtype=like.dtype, device=like.device)
    if tuple(out.shape) != tuple(shape):
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {tuple(shape)}")
    return out


def _check_pair(x: torch.Tensor, q2: torch.Tensor):
    if x.shape != q2.shape or x.dim() != 1:
        raise ValueError("x and q2 must be 1-D tensors of the same length")


def xfxq2(grid: Grid, pid: int, x: torch.Tensor, q2: torch.Tensor, out=None) -> torch.Tensor:
    """x f(x, Q^2) of one flavour (FP64 or FP32 by the input dtype)."""
    _check_pair(x, q2)
    out = _out(out, (x.shape[0],), x)
    lib = _native.load()
    f32 = x.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    fn = lib.xfxq2_f32 if f32 else lib.xfxq2
    check(fn(grid.handle, int(pid), _dev_ptr(x, dt, "x"), _dev_ptr(q2, dt, "q2"), x.shape[0],
             _dev_ptr(out, dt, "out"), _stream_handle(x.device)), "xfxq2")
    return out


def xfxq2_all_flavours(grid: Grid, x: torch.Tensor, q2: torch.Tensor, out=None) -> torch.Tensor:
    """All flavours, [n][nflav] (FP64 or FP32 by the input dtype)."""
    _check_pair(x, q2)
    out = _out(out, (x.shape[0], grid.nflav), x)
    lib = _native.load()
    f32 = x.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    fn = lib.xfxq2_all_flavours_f32 if f32 else lib.xfxq2_all_flavours
    check(fn(grid.handle, _dev_ptr(x, dt, "x"), _dev_ptr(q2, dt, "q2"), x.shape[0],
             _dev_ptr(out, dt, "out"), _stream_handle(x.device)), "xfxq2_all_flavours")
    return out


def xfxq2_all_flavours_alphas(grid: Grid, x: torch.Tensor, q2: torch.Tensor, out=None, alphas_out=None):
    """All flavours [n][nflav] and alpha_s [n] in one pass (FP64 or FP32 by
    the input dtype)."""
    _check_pair(x, q2)
    out = _out(out, (x.shape[0], grid.nflav), x)
    alphas_out = _out(alphas_out, (x.shape[0],), x)
    f32 = x.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    lib = _native.load()
    fn = lib.xfxq2_all_flavours_alphas_f32 if f32 else lib.xfxq2_all_flavours_alphas
    check(fn(grid.handle, _dev_ptr(x, dt, "x"), _dev_ptr(q2, dt, "q2"), x.shape[0], _dev_ptr(out, dt, "out"),
             _dev_ptr(alphas_out, dt, "alphas_out"), _stream_handle(x.device)), "xfxq2_all_flavours_alphas")
    return out, alphas_out


def _lhapdf_paths(set_dir, member: int):
    import os
    d = os.fspath(set_dir).rstrip("/")
    name = os.path.basename(d)
    return os.path.join(d, name + ".info"), os.path.join(d, f"{name}_{member:04d}.dat")


def read_lhapdf(info_path, dat_path) -> dict:
    """Parse one LHAPDF6 member (lhagrid1 text) on the host, with the
    library's own reader: x_knots, nq, q2_knots, pids, values [rows][nx][nflav],
    as_q2, as_vals as numpy arrays."""
    import os
    lib = _native.load()
    h = ctypes.c_void_p(None)
    check(lib.pdf_lhapdf_read(os.fsencode(info_path), os.fsencode(dat_path), ctypes.byref(h)), "pdf_lhapdf_read")
    try:
        d = _native.GridDesc()
        check(lib.pdf_lhapdf_desc(h, ctypes.byref(d)), "pdf_lhapdf_desc")

        def arr(ptr, n, ct):
            return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ct)), shape=(n,)).copy() if n else \
                np.zeros(0, dtype=np.float64 if ct is ctypes.c_double else np.int32)
        nq = arr(d.nq, d.nsub, ctypes.c_int)
        rows = int(nq.sum())
        return {"x_knots": arr(d.x_knots, d.nx, ctypes.c_double), "nq": [int(v) for v in nq],
                "q2_knots": arr(d.q2_knots, rows, ctypes.c_double),
                "pids": [int(v) for v in arr(d.pids, d.nflav, ctypes.c_int)],
                "values": arr(d.values, rows * d.nx * d.nflav, ctypes.c_double).reshape(rows, d.nx, d.nflav),
                "as_q2": arr(d.as_q2, d.na, ctypes.c_double), "as_vals": arr(d.as_vals, d.na, ctypes.c_double)}
    finally:
        lib.pdf_lhapdf_free(h)


def pdf_load_lhapdf(set_dir, member: int = 0, nmem: int = 1) -> Grid:
    """Members member .. member + nmem - 1 of an LHAPDF6 set directory (the
    lhagrid1 text format, read by the library's native reader) onto the
    current CUDA device."""
    import os
    info, dat = _lhapdf_paths(set_dir, member)
    meta = read_lhapdf(info, dat)
    h = ctypes.c_void_p(None)
    dev = torch.device("cuda", torch.cuda.current_device())
    check(_native.load().pdf_load_lhapdf(os.fsencode(os.fspath(set_dir)), int(member), int(nmem), ctypes.byref(h)),
          "pdf_load_lhapdf")
    return Grid(h.value, meta["pids"], dev, len(meta["x_knots"]), len(meta["q2_knots"]), nmem)


class McResult:
    """Sums of a Monte Carlo run and the estimate they give (the mean weight
    and its standard error)."""

    def __init__(self, sums, n):
        self.sum_w, self.sum_w2, self.sum_abs = (float(v) for v in sums)
        self.n = int(n)

    @property
    def estimate(self) -> float:
        return self.sum_w / self.n

    @property
    def std_error(self) -> float:
        m = self.estimate
        var = max(self.sum_w2 / self.n - m * m, 0.0)
        return (var / max(self.n - 1, 1)) ** 0.5

    def __repr__(self):
        return f"McResult(n={self.n}, estimate={self.estimate:.10g} +- {self.std_error:.3g})"


def pdf_mc_integrate(grid: Grid, sqrt_s: float, x_min: float, shat_min: float, seed: int, n_events: int,
                     first_event: int = 0, chunk: int = 1 << 20) -> McResult:
    """Monte Carlo integration of the toy leading-order observable of
    pdf_mc_integrate (include/pdf_gb300.h) over events [first_event,
    first_event + n_events): device RNG, fused PDF + alpha_s load, weights
    summed on the device.  Runs on the grid's device, current stream."""
    cfg = _native.McConfig(float(sqrt_s), float(x_min), float(shat_min), int(seed) & (2**64 - 1))
    sums = (ctypes.c_double * 3)()
    dev = grid.device if isinstance(grid.device, torch.device) else torch.device("cuda", grid.device)
    check(_native.load().pdf_mc_integrate(grid.handle, ctypes.byref(cfg), int(first_event), int(n_events),
                                          int(chunk), sums, _stream_handle(dev)), "pdf_mc_integrate")
    return McResult(sums, n_events)


def xfxq2_all_members(grid: Grid, x: torch.Tensor, q2: torch.Tensor, out=None) -> torch.Tensor:
    """All flavours of every member: [nmem][n][nflav] FP64."""
    _check_pair(x, q2)
    out = _out(out, (grid.nmem, x.shape[0], grid.nflav), x)
    dt = torch.float64
    check(_native.load().xfxq2_all_members(grid.handle, _dev_ptr(x, dt, "x"), _dev_ptr(q2, dt, "q2"), x.shape[0],
                                           _dev_ptr(out, dt, "out"), _stream_handle(x.device)), "xfxq2_all_members")
    return out


def alphas_q2(grid: Grid, q2: torch.Tensor, out=None) -> torch.Tensor:
    """alpha_s(Q^2) (FP64 or FP32 by the input dtype)."""
    if q2.dim() != 1:
        raise ValueError("q2 must be 1-D")
    out = _out(out, (q2.shape[0],), q2)
    lib = _native.load()
    f32 = q2.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    fn = lib.alphas_q2_f32 if f32 else lib.alphas_q2
    check(fn(grid.handle, _dev_ptr(q2, dt, "q2"), q2.shape[0], _dev_ptr(out, dt, "out"),
             _stream_handle(q2.device)), "alphas_q2")
    return out


def alphas_q(grid: Grid, q: torch.Tensor, out=None) -> torch.Tensor:
    """alpha_s at scales Q in GeV (squared by the kernel; FP64 or FP32 by the input dtype)."""
    if q.dim() != 1:
        raise ValueError("q must be 1-D")
    out = _out(out, (q.shape[0],), q)
    lib = _native.load()
    f32 = q.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    fn = lib.alphas_q_f32 if f32 else lib.alphas_q
    check(fn(grid.handle, _dev_ptr(q, dt, "q"), q.shape[0], _dev_ptr(out, dt, "out"),
             _stream_handle(q.device)), "alphas_q")
    return out


def pdf_mc_event(grid: Grid, x1: torch.Tensor, x2: torch.Tensor, s: float, out=None) -> torch.Tensor:
    """Fused Monte Carlo event evaluation: [n][2 nflav + 1] with Q^2 = x1 x2 s."""
    _check_pair(x1, x2)
    out = _out(out, (x1.shape[0], 2 * grid.nflav + 1), x1)
    lib = _native.load()
    f32 = x1.dtype == torch.float32
    dt = torch.float32 if f32 else torch.float64
    fn = lib.pdf_mc_event_f32 if f32 else lib.pdf_mc_event
    check(fn(grid.handle, _dev_ptr(x1, dt, "x1"), _dev_ptr(x2, dt, "x2"), float(s), x1.shape[0],
             _dev_ptr(out, dt, "out"), _stream_handle(x1.device)), "pdf_mc_event")
    return out


def xfxq2_all_flavours_host(grid: Grid, x, q2, out=None, alphas_out=None, with_alphas: bool = False):
    """Host arrays in (numpy or CPU tensors, float64), host [n][nflav] out (and
    alpha_s [n] when with_alphas or alphas_out is given).  Pinned CPU tensors
    give overlapped copies.  Returns out, or (out, alphas_out)."""
    xs = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    qs = q2 if isinstance(q2, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(q2, dtype=np.float64))
    for t, name in ((xs, "x"), (qs, "q2")):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float64 host array")
    if out is None:
        out = torch.empty((xs.shape[0], grid.nflav), dtype=torch.float64)
    if alphas_out is None and with_alphas:
        alphas_out = torch.empty((xs.shape[0],), dtype=torch.float64)
    lib = _native.load()
    aptr = ctypes.c_void_p(alphas_out.data_ptr()) if alphas_out is not None else None
    with torch.cuda.device(grid.device):
        check(lib.xfxq2_all_flavours_host(grid.handle, ctypes.c_void_p(xs.data_ptr()),
                                          ctypes.c_void_p(qs.data_ptr()), xs.shape[0],
                                          ctypes.c_void_p(out.data_ptr()), aptr), "xfxq2_all_flavours_host")
    return out if alphas_out is None else (out, alphas_out)


def set_scratch_limit(nbytes: int):
    """Bound the device scratch one call may take for a sorted path (None: no bound)."""
    lim = (1 << 64) - 1 if nbytes is None else int(nbytes)
    check(_native.load().pdf_set_scratch_limit(lim), "pdf_set_scratch_limit")


def scratch_limit() -> int:
    v = ctypes.c_size_t()
    check(_native.load().pdf_get_scratch_limit(ctypes.byref(v)), "pdf_get_scratch_limit")
    return int(v.value)


def pdf_grid_set_values(grid: Grid, values: torch.Tensor):
    """Replace the grid's knot values ([rows][nx][nflav] float64 CUDA tensor)
    and re-stage its patch coefficients on the current stream."""
    check(_native.load().pdf_grid_set_values(grid.handle, _dev_ptr(values, torch.float64, "values"),
                                             _stream_handle(values.device)), "pdf_grid_set_values")


def xfxq2_all_flavours_vjp(grid: Grid, x: torch.Tensor, q2: torch.Tensor, cot: torch.Tensor,
                           grad_x=None, grad_q2=None, grad_values=None):
    """Gradients of L = sum(cot * xf): fills grad_x [n], grad_q2 [n] (either
    may be None) and accumulates into grad_values [rows][nx][nflav] (None to
    skip).  Returns (grad_x, grad_q2, grad_values)."""
    _check_pair(x, q2)
    if tuple(cot.shape) != (x.shape[0], grid.nflav):
        raise ValueError(f"cot must be [n][nflav], got {tuple(cot.shape)}")
    dt = torch.float64
    opt = lambda t, name: _dev_ptr(t, dt, name) if t is not None else None  # noqa: E731
    check(_native.load().xfxq2_all_flavours_vjp(
        grid.handle, _dev_ptr(x, dt, "x"), _dev_ptr(q2, dt, "q2"), x.shape[0], _dev_ptr(cot, dt, "cot"),
        opt(grad_x, "grad_x"), opt(grad_q2, "grad_q2"), opt(grad_values, "grad_values"),
        _stream_handle(x.device)), "xfxq2_all_flavours_vjp")
    return grad_x, grad_q2, grad_values


class XfxQ2AllFlavours(torch.autograd.Function):
    """xf for all flavours, differentiable in x, Q^2 and the knot values.

    forward(grid, x, q2, values): if `values` is given it is staged into the
    grid first (so the output is a function of it); backward runs the
    library's adjoint kernel."""

    @staticmethod
    def forward(ctx, grid, x, q2, values):
        if values is not None:
            pdf_grid_set_values(grid, values.detach())
        out = xfxq2_all_flavours(grid, x.detach(), q2.detach())
        ctx.grid = grid
        ctx.vshape = None if values is None else tuple(values.shape)
        ctx.save_for_backward(x, q2)
        return out

    @staticmethod
    def backward(ctx, gout):
        x, q2 = ctx.saved_tensors
        _, nx, nq, nv = ctx.needs_input_grad
        gx = torch.empty_like(x) if nx else None
        gq = torch.empty_like(q2) if nq else None
        gv = torch.zeros(ctx.vshape, dtype=torch.float64, device=x.device) if (nv and ctx.vshape) else None
        xfxq2_all_flavours_vjp(ctx.grid, x.detach(), q2.detach(), gout.contiguous(), gx, gq, gv)
        return None, gx, gq, gv


def xfxq2_all_flavours_diff(grid: Grid, x: torch.Tensor, q2: torch.Tensor, values: torch.Tensor = None):
    """Differentiable all-flavour evaluation (see XfxQ2AllFlavours)."""
    return XfxQ2AllFlavours.apply(grid, x, q2, values)
