"""ctypes binding of libpdfgb300.so (the C ABI declared in include/pdf_gb300.h).

Argument marshalling only: every evaluation runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library cannot be loaded or a
call fails, a PdfError is raised.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libpdfgb300.so"
HEADERS = sorted((_PKG.parent / "include").glob("*.h"))
# measurement and test hooks: a library of their own, not the C ABI above
PROBE_LIB_PATH = _PKG / "_lib" / "libpdfgb300_probe.so"
PROBE_HEADERS = sorted((_PKG / "probe").glob("*.h"))

PDF_OK = 0
ERRORS = {
    -1: "PDF_ERR_NULL", -2: "PDF_ERR_GRID", -3: "PDF_ERR_PID", -4: "PDF_ERR_CUDA",
    -5: "PDF_ERR_ALLOC", -6: "PDF_ERR_ARG", -7: "PDF_ERR_NO_ALPHAS",
}


class PdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("x_knots", ctypes.c_void_p),
        ("nsub", ctypes.c_int), ("nq", ctypes.c_void_p),
        ("q2_knots", ctypes.c_void_p),
        ("nflav", ctypes.c_int), ("pids", ctypes.c_void_p),
        ("values", ctypes.c_void_p),
        ("na", ctypes.c_int), ("as_q2", ctypes.c_void_p), ("as_vals", ctypes.c_void_p),
    ]


_lib = None
_lock = threading.Lock()

P, SZ, I32, F64, F32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double, ctypes.c_float
SIGNATURES = {
    "pdf_load_grid": (I32, [ctypes.POINTER(GridDesc), ctypes.POINTER(P)]),
    "pdf_free_grid": (I32, [P]),
    "pdf_grid_nflav": (I32, [P]),
    "pdf_load_grid_members": (I32, [ctypes.POINTER(GridDesc), I32, P, ctypes.POINTER(P)]),
    "pdf_grid_nmembers": (I32, [P]),
    "xfxq2_all_members": (I32, [P, P, P, SZ, P, P]),
    "pdf_grid_pid_column": (I32, [P, I32]),
    "xfxq2": (I32, [P, I32, P, P, SZ, P, P]),
    "xfxq2_all_flavours": (I32, [P, P, P, SZ, P, P]),
    "xfxq2_all_flavours_alphas": (I32, [P, P, P, SZ, P, P, P]),
    "xfxq2_all_flavours_alphas_f32": (I32, [P, P, P, SZ, P, P, P]),
    "pdf_mc_integrate": (I32, [P, P, ctypes.c_ulonglong, ctypes.c_ulonglong, SZ, P, P]),
    "pdf_load_lhapdf": (I32, [ctypes.c_char_p, I32, I32, ctypes.POINTER(P)]),
    "pdf_lhapdf_read": (I32, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(P)]),
    "pdf_lhapdf_desc": (I32, [P, ctypes.POINTER(GridDesc)]),
    "pdf_lhapdf_free": (I32, [P]),
    "alphas_q2": (I32, [P, P, SZ, P, P]),
    "xfxq2_f32": (I32, [P, I32, P, P, SZ, P, P]),
    "xfxq2_all_flavours_f32": (I32, [P, P, P, SZ, P, P]),
    "alphas_q2_f32": (I32, [P, P, SZ, P, P]),
    "alphas_q": (I32, [P, P, SZ, P, P]),
    "alphas_q_f32": (I32, [P, P, SZ, P, P]),
    "pdf_mc_event": (I32, [P, P, P, F64, SZ, P, P]),
    "pdf_mc_event_f32": (I32, [P, P, P, F32, SZ, P, P]),
    "xfxq2_all_flavours_host": (I32, [P, P, P, SZ, P, P]),
    "xfxq2_all_flavours_host_noalloc": (I32, [P, P, P, SZ, P, P, P]),
    "xfxq2_all_flavours_vjp": (I32, [P, P, P, SZ, P, P, P, P, P]),
    "pdf_grid_set_values": (I32, [P, P, P]),
    "pdf_grid_invalid_count": (I32, [P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "pdf_grid_reset_invalid_count": (I32, [P]),
    "pdf_last_error": (ctypes.c_char_p, []),
    "pdf_set_scratch_limit": (I32, [SZ]),
    "pdf_get_scratch_limit": (I32, [ctypes.POINTER(SZ)]),
    "pdf_surrogate_create": (I32, [P, P, P, I32, ctypes.POINTER(P)]),
    "pdf_surrogate_create_ex": (I32, [P, P, P, I32, I32, ctypes.POINTER(P)]),
    "pdf_surrogate_free": (I32, [P]),
    "pdf_surrogate_nparams": (I32, [P, ctypes.POINTER(SZ)]),
    "pdf_surrogate_get_params": (I32, [P, P]),
    "pdf_surrogate_set_params": (I32, [P, P]),
    "pdf_surrogate_loss_grad": (I32, [P, P, P, P, SZ, ctypes.POINTER(ctypes.c_double), P]),
    "pdf_surrogate_trace": (I32, [P, I32, I32, P]),
    "pdf_surrogate_map": (I32, [P, P]),
    "pdf_surrogate_train": (I32, [P, P, P, P, SZ, P, ctypes.POINTER(ctypes.c_double), P]),
    "pdf_surrogate_eval": (I32, [P, P, P, SZ, P, P]),
    "pdf_surrogate_build_error_map": (I32, [P, P, P, P, SZ, F64, P]),
    "pdf_surrogate_eval_fallback": (I32, [P, P, P, P, SZ, P, ctypes.POINTER(ctypes.c_ulonglong), P]),
}


class McConfig(ctypes.Structure):
    _fields_ = [("sqrt_s", ctypes.c_double), ("x_min", ctypes.c_double), ("shat_min", ctypes.c_double),
                ("seed", ctypes.c_ulonglong)]


class TrainConfig(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("steps", ctypes.c_int), ("lr", ctypes.c_float),
                ("lr_min", ctypes.c_float), ("warmup", ctypes.c_int)]


PROBE_SIGNATURES = {
    "pdf_probe_fma_rate": (I32, [I32, I32, ctypes.POINTER(ctypes.c_double)]),
    "pdf_probe_math": (I32, [P, I32, P, P, SZ, P, P]),
    "pdf_probe_last_error": (ctypes.c_char_p, []),
}


def header_functions(headers=None) -> list[str]:
    """Names of the functions the headers (default: those under include/) declare."""
    names = []
    for h in HEADERS if headers is None else headers:
        names += re.findall(r"^PDF_API\s+(?:const\s+char\s*\*|int)\s*([A-Za-z_0-9]+)\s*\(", h.read_text(),
                            flags=re.M)
    return names


def load(build_if_missing: bool = True):
    """Load the library (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not LIB_PATH.exists():
            if not build_if_missing:
                raise PdfError(-4, f"CUDA library not built: {LIB_PATH}")
            from . import build as _build

            _build.build()
        lib = ctypes.CDLL(str(LIB_PATH), mode=os.RTLD_LOCAL if hasattr(os, "RTLD_LOCAL") else 0)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


_probe = None


def load_probe():
    """The measurement/test hooks library (built beside the evaluation library)."""
    global _probe
    with _lock:
        if _probe is not None:
            return _probe
        if not PROBE_LIB_PATH.exists():
            from . import build as _build

            _build.build()
        lib = ctypes.CDLL(str(PROBE_LIB_PATH), mode=os.RTLD_LOCAL if hasattr(os, "RTLD_LOCAL") else 0)
        for name, (res, args) in PROBE_SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _probe = lib
        return lib


def check_probe(rc: int, what: str):
    if rc != PDF_OK:
        raise PdfError(rc, f"{what}: {load_probe().pdf_probe_last_error().decode()}")


def last_error() -> str:
    return load().pdf_last_error().decode()


def check(rc: int, what: str):
    if rc != PDF_OK:
        raise PdfError(rc, f"{what}: {last_error()}")
