"""The no-allocation host entry point, called through the C ABI.

xfxq2_all_flavours_host_noalloc serves callers that cannot let the library
allocate device memory (an integrator calling the PDF inside its own loop,
where a cudaMalloc would synchronise the device; a program whose device
memory belongs to another pool).  It stages through a fixed array in the
library instead of buffers the grid allocates.  Here it must give the same
results as the existing host entry point, on two calls in a row (the shared
array keeps the first call's contents), and reject a batch larger than the
array.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from parity import RTOL_FP64, scaled_err

pytestmark = pytest.mark.gpu


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def test_no_alloc_entry_matches_host_entry_on_two_calls(synth):
    import paper_2009_06635_gb300 as P
    from paper_2009_06635_gb300 import _native

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    lib = _native.load()
    g = synth.grid_full()
    G = P.pdf_load_grid(g)
    cap = (1 << 21) // (3 + g.nflav)
    stream = ctypes.c_void_p(0)
    # two different batches, the second shorter than the first
    for n, seed in ((cap, 3), (cap // 3 + 7, 41)):
        x, q2 = synth.queries_full(n, seed)
        want, want_a = P.xfxq2_all_flavours_host(G, x, q2, with_alphas=True)
        want, want_a = want.numpy(), want_a.numpy()
        out = np.full((n, g.nflav), np.nan)
        a = np.full(n, np.nan)
        rc = lib.xfxq2_all_flavours_host_noalloc(G.handle, _ptr(x), _ptr(q2), n, _ptr(out), _ptr(a), stream)
        assert rc == 0, _native.last_error()
        assert np.array_equal(np.isnan(out), np.isnan(want))
        ok = ~np.isnan(want)
        assert (scaled_err(out[ok], want[ok], np.abs(want[ok])) <= RTOL_FP64).all()
        assert (scaled_err(a, want_a, np.abs(want_a)) <= RTOL_FP64).all()
    # a batch larger than the fixed array is refused, and says why
    big = cap + 1
    x, q2 = synth.queries_full(big, 5)
    out = np.empty((big, g.nflav))
    rc = lib.xfxq2_all_flavours_host_noalloc(G.handle, _ptr(x), _ptr(q2), big, _ptr(out), None, stream)
    assert rc == -6
    assert "capacity" in _native.last_error()
