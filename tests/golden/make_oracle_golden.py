"""Writes oracle_regression.txt: oracle values on a few seeded points of the
single-subgrid and three-subgrid workloads (in-grid and extrapolated).  The
paper prints no worked example, so these values come from the oracle alone
and guard it against unintended changes.  Run: python tests/golden/make_oracle_golden.py"""
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2009_06635_gb300 import synthetic as S  # noqa: E402

OUT = Path(__file__).with_name("oracle_regression.txt")


def cases():
    yield "single_subgrid", S.grid_single_subgrid(), S.queries_single_subgrid(24, 2)
    yield "three_subgrids", S.grid_full(), S.queries_full(48, 3)


def main():
    lines = ["# name point x q2 alphas xf[0..nflav)"]
    for name, g, (x, q2) in cases():
        og = oracle.OracleGrid(g)
        v, _, _ = og.xfxq2(x, q2)
        a, _ = og.alphas(q2)
        for p in range(len(x)):
            vals = " ".join(f"{t:.17g}" for t in v[p])
            lines.append(f"{name} {p} {x[p]:.17g} {q2[p]:.17g} {a[p]:.17g} {vals}")
    OUT.write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
