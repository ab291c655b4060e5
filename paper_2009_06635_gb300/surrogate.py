"""Python binding of the learned surrogate (include/pdf_surrogate.h).

    s = Surrogate(grid)                      # seeded initial parameters
    s.train(grid, x, q2, batch=8192, steps=4000)
    stats = s.build_error_map(grid, xv, qv, threshold=1e-3)
    out, n_fb = s.eval_fallback(grid, x, q2)  # network where accepted, interpolator elsewhere
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native, synthetic
from ._native import PdfError, check
from .pdf import Grid, _dev_ptr, _stream_handle


class Surrogate:
    TARGETS = {"asinh": 0, "envelope": 1, "residual": 2}  # PDF_SURR_ASINH, _ENVELOPE, _RESIDUAL

    def __init__(self, grid: Grid, params=None, freq=None, max_batch: int = 16384, seed: int = 9,
                 target: str = "asinh"):
        if params is None or freq is None:
            p0, f0 = synthetic.surrogate_init(grid.nflav, seed)
            params = p0 if params is None else params
            freq = f0 if freq is None else freq
        p = np.ascontiguousarray(params, dtype=np.float32)
        f = np.ascontiguousarray(freq, dtype=np.float32)
        h = ctypes.c_void_p(None)
        with torch.cuda.device(grid.device):
            check(_native.load().pdf_surrogate_create_ex(grid.handle, p.ctypes.data, f.ctypes.data, int(max_batch),
                                                         self.TARGETS[target], ctypes.byref(h)),
                  "pdf_surrogate_create")
        self.target = target
        self._h = h
        self.nflav = grid.nflav
        self.max_batch = max_batch
        self.device = grid.device

    @property
    def handle(self):
        if not self._h:
            raise PdfError(-1, "surrogate has been freed")
        return self._h

    def free(self):
        if self._h:
            _native.load().pdf_surrogate_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def nparams(self) -> int:
        n = ctypes.c_size_t(0)
        check(_native.load().pdf_surrogate_nparams(self.handle, ctypes.byref(n)), "pdf_surrogate_nparams")
        return int(n.value)

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        check(_native.load().pdf_surrogate_get_params(self.handle, out.ctypes.data), "pdf_surrogate_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(_native.load().pdf_surrogate_set_params(self.handle, p.ctypes.data), "pdf_surrogate_set_params")

    def loss_grad(self, x: torch.Tensor, q2: torch.Tensor, xf: torch.Tensor):
        """One forward/backward on a batch with given target values xf [n][nflav]."""
        loss = ctypes.c_double(0.0)
        grad = np.empty(self.nparams, dtype=np.float32)
        check(_native.load().pdf_surrogate_loss_grad(
            self.handle, _dev_ptr(x, torch.float64, "x"), _dev_ptr(q2, torch.float64, "q2"),
            _dev_ptr(xf, torch.float64, "xf"), x.shape[0], ctypes.byref(loss), grad.ctypes.data),
            "pdf_surrogate_loss_grad")
        return loss.value, grad

    def trace(self, what: str, layer: int = 0, n: int = None) -> np.ndarray:
        """An intermediate of the last loss_grad pass: "h" (bfloat16 activations),
        "z" (pre-activations), "g" (backward signals), "y" (outputs), "t" (targets)."""
        code = {"h": 0, "z": 1, "g": 2, "y": 3, "t": 4}[what]
        cols = {"h": 32 if layer == 0 else 128, "z": 128, "g": 16 if layer == 4 else 128, "y": 16, "t": 16}[what]
        out = np.empty((n, cols), dtype=np.float32)
        check(_native.load().pdf_surrogate_trace(self.handle, code, int(layer), out.ctypes.data), "pdf_surrogate_trace")
        return out

    def train(self, grid: Grid, x: torch.Tensor, q2: torch.Tensor, batch: int = 8192, steps: int = 1000,
              lr: float = 2e-3, lr_min: float = 2e-5, warmup: int = 100) -> float:
        cfg = _native.TrainConfig(int(batch), int(steps), float(lr), float(lr_min), int(warmup))
        loss = ctypes.c_double(0.0)
        check(_native.load().pdf_surrogate_train(
            self.handle, grid.handle, _dev_ptr(x, torch.float64, "x"), _dev_ptr(q2, torch.float64, "q2"),
            x.shape[0], ctypes.byref(cfg), ctypes.byref(loss), _stream_handle(x.device)), "pdf_surrogate_train")
        return loss.value

    def eval(self, x: torch.Tensor, q2: torch.Tensor, out=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((x.shape[0], self.nflav), dtype=torch.float32, device=x.device)
        check(_native.load().pdf_surrogate_eval(
            self.handle, _dev_ptr(x, torch.float64, "x"), _dev_ptr(q2, torch.float64, "q2"), x.shape[0],
            _dev_ptr(out, torch.float32, "out"), _stream_handle(x.device)), "pdf_surrogate_eval")
        return out

    def build_error_map(self, grid: Grid, x: torch.Tensor, q2: torch.Tensor, threshold: float = 1e-3) -> dict:
        st = np.zeros(4)
        check(_native.load().pdf_surrogate_build_error_map(
            self.handle, grid.handle, _dev_ptr(x, torch.float64, "x"), _dev_ptr(q2, torch.float64, "q2"),
            x.shape[0], float(threshold), st.ctypes.data), "pdf_surrogate_build_error_map")
        m = self.tile_map()
        return {"tiles_accepted": int(st[0]), "tiles_sampled": int(st[1]), "max_error": float(st[2]),
                "median_tile_error": float(st[3]), "threshold": threshold, "tiles_network": int((m == 1).sum()),
                "tiles_base_only": int((m == 2).sum())}

    def tile_map(self) -> np.ndarray:
        """The last error map's tile states [64 (z1 tiles)][64 (z0 tiles)]: 0 the
        interpolator, 1 the network, 2 the residual target's base alone."""
        m = np.zeros(64 * 64, dtype=np.uint8)
        check(_native.load().pdf_surrogate_map(self.handle, m.ctypes.data), "pdf_surrogate_map")
        return m.reshape(64, 64)

    def eval_fallback(self, grid: Grid, x: torch.Tensor, q2: torch.Tensor, out=None):
        if out is None:
            out = torch.empty((x.shape[0], self.nflav), dtype=torch.float64, device=x.device)
        nfb = ctypes.c_ulonglong(0)
        check(_native.load().pdf_surrogate_eval_fallback(
            self.handle, grid.handle, _dev_ptr(x, torch.float64, "x"), _dev_ptr(q2, torch.float64, "q2"),
            x.shape[0], _dev_ptr(out, torch.float64, "out"), ctypes.byref(nfb), _stream_handle(x.device)),
            "pdf_surrogate_eval_fallback")
        return out, int(nfb.value)
