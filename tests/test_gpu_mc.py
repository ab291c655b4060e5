"""Monte Carlo integration on the device (PDFFlow Sec. 4.1's PDF load inside
a VegasFlow-style loop, Sec. 5): device-generated events, the fused event
kernel, weights summed on the device -- against the oracle's sums over the
same events, plus reproducibility, chunking and additivity."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2009_06635_gb300")

CFG = dict(sqrt_s=13000.0, x_min=1e-6, shat_min=100.0, seed=2024)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def full(synth, oracle_mod):
    g = synth.grid_full()
    return g, P.pdf_load_grid(g), oracle_mod.OracleGrid(g)


def run(G, n, first=0, chunk=1 << 20, **kw):
    c = dict(CFG, **kw)
    return P.pdf_mc_integrate(G, c["sqrt_s"], c["x_min"], c["shat_min"], c["seed"], n, first_event=first, chunk=chunk)


def test_sums_match_the_oracle_over_the_same_events(full):
    from oracle import mc
    g, G, og = full
    first, n = 12_345, 60_001
    r = run(G, n, first=first, chunk=16_384)  # four chunks, the last one ragged
    w = mc.weights(og, g.pids, CFG["sqrt_s"], CFG["x_min"], CFG["shat_min"], CFG["seed"], first, n, g.x_knots[-1])
    sw, sw2, sa = mc.sums(w)
    assert np.count_nonzero(w) > 0.5 * n
    assert abs(r.sum_w - sw) <= 1e-12 * sa, (r.sum_w, sw)
    assert abs(r.sum_abs - sa) <= 1e-12 * sa
    assert abs(r.sum_w2 - sw2) <= 1e-12 * sw2
    assert r.n == n and np.isfinite(r.std_error) and r.std_error > 0


@pytest.mark.parametrize("kw", [{}, dict(sqrt_s=2e5, x_min=1e-10, shat_min=0.5)],
                         ids=["inside_the_grid", "continued_events"])
def test_two_launch_chunks_match_the_oracle(full, kw):
    """Chunks of 65536 events or more take the near and far launches; events
    below the s-hat cut are not evaluated, and where no evaluated event can
    leave the grid (the standard configuration: x_min above the first x
    knot, x_max^2 s below Q2max, shat_min above Q2min) the far launch is left
    out.  The other configuration has evaluated events below x0, above
    Q2max and below Q2min."""
    from oracle import mc
    g, G, og = full
    c = dict(CFG, **kw)
    first, n = 777, 70_001
    r = run(G, n, first=first, chunk=n, **kw)
    w = mc.weights(og, g.pids, c["sqrt_s"], c["x_min"], c["shat_min"], c["seed"], first, n, g.x_knots[-1])
    sw, sw2, sa = mc.sums(w)
    assert np.count_nonzero(w) > 0.3 * n
    assert abs(r.sum_w - sw) <= 1e-12 * sa, (r.sum_w, sw)
    assert abs(r.sum_abs - sa) <= 1e-12 * sa
    assert abs(r.sum_w2 - sw2) <= 1e-12 * sw2
    if kw:  # the events do leave the grid
        x1, x2 = mc.events(c["seed"], first, n, c["x_min"], g.x_knots[-1])
        q2 = x1 * x2 * c["sqrt_s"] ** 2
        kept = q2 >= c["shat_min"]
        assert (kept & (np.minimum(x1, x2) < g.x_knots[0])).any()
        assert (kept & (q2 > g.q2_knots[-1])).any() and (kept & (q2 < g.q2_knots[0])).any()


def test_reproducible_and_chunking_changes_only_rounding(full):
    g, G, og = full
    n = 300_007
    a = run(G, n, chunk=65_536)
    b = run(G, n, chunk=65_536)
    assert (a.sum_w, a.sum_w2, a.sum_abs) == (b.sum_w, b.sum_w2, b.sum_abs)
    c = run(G, n, chunk=n)
    assert abs(a.sum_w - c.sum_w) <= 1e-13 * a.sum_abs
    # sums over consecutive ranges add up
    k = 123_456
    lo, hi = run(G, k, chunk=50_000), run(G, n - k, first=k, chunk=50_000)
    assert abs(lo.sum_w + hi.sum_w - a.sum_w) <= 1e-13 * a.sum_abs
    # a different seed gives a different but statistically compatible estimate
    d = run(G, n, chunk=65_536, seed=7)
    assert d.sum_w != a.sum_w
    assert abs(d.estimate - a.estimate) < 6 * np.hypot(a.std_error, d.std_error)


def test_rejected_arguments(full, synth):
    g, G, og = full
    with pytest.raises(P.PdfError):
        run(G, 10, x_min=0.0)
    with pytest.raises(P.PdfError):
        run(G, 10, x_min=2.0)
    with pytest.raises(P.PdfError):
        run(G, 10, chunk=0)
    g1 = synth.grid_single_subgrid()  # flavours -5..5 and the gluon, with alpha_s
    r = run(P.pdf_load_grid(g1), 1000)
    assert np.isfinite(r.sum_w)
    no_as = P.pdf_load_grid(x_knots=g1.x_knots, nq=g1.nq, q2_knots=g1.q2_knots, pids=g1.pids, values=g1.values)
    with pytest.raises(P.PdfError):
        run(no_as, 10)
