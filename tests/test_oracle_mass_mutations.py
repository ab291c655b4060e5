"""The data-mass pins catch plausible mistakes in the oracle's s arithmetic.

Each case plants one mistake in a private copy of the oracle's C source (on
the CPU, in a temporary directory), builds it, and checks that at least one
pin of test_oracle_mass_pins fails against the planted copy.  The committed
oracle is untouched.
"""
import importlib.util
import shutil
import sys
from pathlib import Path

import pytest

import test_oracle_mass_pins as pins

ROOT = Path(__file__).resolve().parents[1]

MUTATIONS = {
    "mass scaled by 10": ("num r = {c, 0.0, 0.0, fabs(c)};", "num r = {c, 0.0, 0.0, 10.0 * fabs(c)};"),
    "product drops a term": ("r.s = fabs(b.v) * a.s + fabs(a.v) * b.s;", "r.s = fabs(a.v) * b.s;"),
    "difference cancels": ("r.d = a.d - b.d; r.m = a.m + b.m + fabs(r.v); r.s = a.s + b.s;",
                           "r.d = a.d - b.d; r.m = a.m + b.m + fabs(r.v); r.s = fabs(a.s - b.s);"),
    "quotient drops the divisor's mass": ("r.s = (a.s + fabs(r.v) * b.s) / fabs(b.v);", "r.s = a.s / fabs(b.v);"),
}

PINS = [pins.test_constant_grid_mass_matches_closed_form, pins.test_mass_bounds_on_a_general_grid,
        pins.test_pair_rule_mass_at_knot_sites, pins.test_linear_branch_mass, pins.test_low_q2_rule_mass,
        pins.test_alphas_mass_constant_nodes]


def _planted_oracle(tmp: Path, name: str, old: str, new: str):
    d = tmp / f"oracle_{abs(hash(name)) % 10**8}"
    shutil.copytree(ROOT / "oracle", d, ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    src = d / "pdf_oracle.c"
    text = src.read_text()
    assert text.count(old) == 1, f"mutation site not found: {old}"
    src.write_text(text.replace(old, new))
    spec = importlib.util.spec_from_file_location(d.name, d / "__init__.py", submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[d.name] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_planted_mass_mistake_fails_a_pin(name, tmp_path, synth):
    old, new = MUTATIONS[name]
    mod = _planted_oracle(tmp_path, name, old, new)
    failed = []
    for pin in PINS:
        try:
            pin(mod, synth)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake '{name}'"
