"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/pdf_gb300.h declares, and rejects malformed
descriptors and NULL arguments on the host (validation precedes any CUDA call)."""
import ctypes
import subprocess

import numpy as np
import pytest

from paper_2009_06635_gb300 import _native, synthetic


@pytest.fixture(scope="module")
def lib():
    return _native.load()


def test_library_exports_every_declared_function(lib):
    names = _native.header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_native.SIGNATURES), set(names) ^ set(_native.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", str(_native.LIB_PATH)], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported


def test_probe_hooks_live_in_their_own_library(lib):
    """The measurement/test hooks are a separate library: the evaluation
    library exports none of them, the probe library exports what its header
    declares."""
    out = subprocess.run(["nm", "-D", "--defined-only", str(_native.LIB_PATH)], capture_output=True, text=True).stdout
    assert not [l for l in out.splitlines() if "pdf_probe" in l]
    probe = _native.load_probe()
    names = _native.header_functions(_native.PROBE_HEADERS)
    assert set(names) == set(_native.PROBE_SIGNATURES)
    for n in names:
        assert hasattr(probe, n), n
    assert probe.pdf_probe_fma_rate(16, 10, None) == -1  # NULL output checked before any CUDA call
    assert b"NULL" in probe.pdf_probe_last_error()


def test_scratch_limit_round_trip(lib):
    import paper_2009_06635_gb300 as P

    before = P.scratch_limit()
    try:
        P.set_scratch_limit(12345)
        assert P.scratch_limit() == 12345
        P.set_scratch_limit(None)
        assert P.scratch_limit() == (1 << 64) - 1
    finally:
        P.set_scratch_limit(before)
    assert lib.pdf_get_scratch_limit(None) == -1


def _desc(g, **over):
    arrs = dict(x=np.ascontiguousarray(g.x_knots), nq=np.ascontiguousarray(g.nq, dtype=np.int32),
                q2=np.ascontiguousarray(g.q2_knots), pids=np.ascontiguousarray(g.pids, dtype=np.int32),
                vals=np.ascontiguousarray(g.values), aq=np.ascontiguousarray(g.as_q2),
                av=np.ascontiguousarray(g.as_vals))
    arrs.update(over)
    d = _native.GridDesc(len(arrs["x"]), arrs["x"].ctypes.data, len(arrs["nq"]), arrs["nq"].ctypes.data,
                         arrs["q2"].ctypes.data, len(arrs["pids"]), arrs["pids"].ctypes.data,
                         arrs["vals"].ctypes.data, len(arrs["aq"]), arrs["aq"].ctypes.data,
                         arrs["av"].ctypes.data)
    return d, arrs


def _load(lib, d):
    h = ctypes.c_void_p(None)
    rc = lib.pdf_load_grid(ctypes.byref(d), ctypes.byref(h))
    return rc, h


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p(None)
    assert lib.pdf_load_grid(None, ctypes.byref(h)) == -1
    assert b"NULL" in lib.pdf_last_error()
    assert lib.xfxq2_all_flavours(None, None, None, 10, None, None) == -1
    assert lib.alphas_q2(None, None, 0, None, None) == -1
    assert lib.alphas_q(None, None, 0, None, None) == -1
    assert b"alphas_q" in lib.pdf_last_error()
    assert lib.alphas_q_f32(None, None, 0, None, None) == -1
    assert lib.xfxq2(None, 21, None, None, 0, None, None) == -1
    assert lib.pdf_mc_event(None, None, None, 1.0, 0, None, None) == -1
    assert lib.xfxq2_all_flavours_host(None, None, None, 0, None, None) == -1
    assert lib.pdf_free_grid(None) == 0
    c = ctypes.c_ulonglong()
    assert lib.pdf_grid_invalid_count(None, ctypes.byref(c)) == -1


def test_null_arguments_of_the_growth_entries_are_rejected(lib):
    """The adjoint, member sets, Monte Carlo integration, surrogate and LHAPDF
    entries validate their handles before any CUDA call, and freeing NULL is
    a no-op."""
    h = ctypes.c_void_p(None)
    assert lib.xfxq2_all_flavours_vjp(None, None, None, 10, None, None, None, None, None) == -1
    assert b"vjp" in lib.pdf_last_error()
    assert lib.xfxq2_all_members(None, None, None, 10, None, None) == -1
    assert lib.pdf_mc_integrate(None, None, 0, 10, 10, None, None) == -1
    assert lib.pdf_surrogate_create(None, None, None, 1024, ctypes.byref(h)) == -1
    assert lib.pdf_surrogate_create_ex(None, None, None, 1024, 0, ctypes.byref(h)) == -1
    assert lib.pdf_surrogate_eval(None, None, None, 10, None, None) == -1
    assert lib.pdf_surrogate_train(None, None, None, None, 10, None, None, None) == -1
    assert lib.pdf_surrogate_build_error_map(None, None, None, None, 10, 1e-3, None) == -1
    nfb = ctypes.c_ulonglong()
    assert lib.pdf_surrogate_eval_fallback(None, None, None, None, 10, None, ctypes.byref(nfb), None) == -1
    n = ctypes.c_size_t()
    assert lib.pdf_surrogate_nparams(None, ctypes.byref(n)) == -1
    assert lib.pdf_surrogate_free(None) == 0
    assert lib.pdf_lhapdf_read(None, None, ctypes.byref(h)) == -1
    assert lib.pdf_load_lhapdf(None, 0, 1, ctypes.byref(h)) == -1
    assert lib.pdf_lhapdf_free(None) == 0
    assert h.value is None


@pytest.mark.parametrize("case", ["x_not_increasing", "x_above_one", "x_zero", "nq_one", "boundary_gap",
                                  "q2_negative", "value_nan", "pid_repeat", "alphas_decreasing",
                                  "alphas_short_subgrid", "nx_one"])
def test_malformed_descriptors_are_rejected(lib, case):
    g = synthetic.grid_single_subgrid()
    x = g.x_knots.copy()
    over = {}
    if case == "x_not_increasing":
        x[5] = x[4]
        over["x"] = x
    elif case == "x_above_one":
        x[-1] = 1.5
        over["x"] = x
    elif case == "x_zero":
        x[0] = 0.0
        over["x"] = x
    elif case == "nq_one":
        over["nq"] = np.array([1, 39], dtype=np.int32)
    elif case == "boundary_gap":
        q2 = g.q2_knots.copy()
        over["nq"] = np.array([20, 20], dtype=np.int32)
        over["q2"] = q2
    elif case == "q2_negative":
        q2 = g.q2_knots.copy()
        q2[0] = -1.0
        over["q2"] = q2
    elif case == "value_nan":
        v = g.values.copy()
        v[3, 4, 1] = np.nan
        over["vals"] = v
    elif case == "pid_repeat":
        p = np.array(g.pids, dtype=np.int32)
        p[1] = p[0]
        over["pids"] = p
    elif case == "alphas_decreasing":
        aq = g.as_q2.copy()
        aq[3], aq[4] = aq[4], aq[3]
        over["aq"] = aq
    elif case == "alphas_short_subgrid":
        aq = g.as_q2.copy()
        aq[1] = aq[0]
        over["aq"] = aq
    elif case == "nx_one":
        over["x"] = x[:1]
    d, keep = _desc(g, **over)
    rc, h = _load(lib, d)
    assert rc == -2, (case, rc, lib.pdf_last_error())
    assert not h.value
    assert lib.pdf_last_error()


def test_python_binding_names_match_the_c_abi():
    import paper_2009_06635_gb300 as P

    for name in ("pdf_load_grid", "xfxq2", "xfxq2_all_flavours", "alphas_q2", "alphas_q", "pdf_mc_event",
                 "xfxq2_all_flavours_host"):
        assert callable(getattr(P, name))
        assert name in _native.SIGNATURES
