"""Host-side helpers of bench.py: the share of Monte Carlo events that pass
the s-hat cut (the integration leg counts only the evaluations it makes)
against the oracle's own event generator, and the source closure that
decides whether a committed ncu capture still describes a kernel."""
import math

import numpy as np
import pytest

bench = pytest.importorskip("bench")
mc = pytest.importorskip("oracle.mc")


@pytest.mark.parametrize("shat_min", [1.0, 100.0, 1e4, 1e6, 1e8])
def test_cut_pass_fraction_matches_the_generated_events(shat_min):
    s, x_min, x_max, n = 13000.0 ** 2, 1e-6, 1.0, 400_000
    x1, x2 = mc.events(4, 0, n, x_min, x_max)
    seen = np.mean(x1 * x2 * s >= shat_min)
    want = bench.mc_cut_pass_fraction(x_min, x_max, s, shat_min)
    sigma = math.sqrt(max(want * (1 - want), 1e-12) / n)
    assert abs(seen - want) <= 5 * sigma + 1e-6, (seen, want)


def test_cut_pass_fraction_limits():
    s = 13000.0 ** 2
    assert bench.mc_cut_pass_fraction(1e-6, 1.0, s, 0.0) == 1.0
    assert bench.mc_cut_pass_fraction(1e-6, 1.0, s, 1e-12 * s) == 1.0  # below x_min^2 s
    assert bench.mc_cut_pass_fraction(1e-6, 1.0, s, s) == 0.0
    # the two branches of the triangular density meet at ln x1 + ln x2 = lo + hi
    mid = math.exp(math.log(1e-6) + math.log(1.0)) * s
    a = bench.mc_cut_pass_fraction(1e-6, 1.0, s, mid * (1 - 1e-12))
    b = bench.mc_cut_pass_fraction(1e-6, 1.0, s, mid * (1 + 1e-12))
    assert abs(a - 0.5) < 1e-9 and abs(b - 0.5) < 1e-9


def test_capture_hash_follows_the_includes():
    files = {p.name for p in bench.kernel_source_files("k_xf64<points> near + far")}
    # the translation unit, the table staging, and what they include
    assert {"xf64.cu", "grid.cu", "sites.cuh", "ffpos.cuh", "ffmath.cuh", "ff.cuh", "tang.cuh"} <= files
    files32 = {p.name for p in bench.kernel_source_files("k_xf32<points>")}
    assert {"xfxq2.cu", "sites.cuh", "pdf_internal.cuh"} <= files32 and "xf64.cu" not in files32
