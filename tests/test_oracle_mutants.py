"""Plant plausible mistakes in copies of the oracle and check that the pins catch each.

Each mutant is a textual edit of ``oracle/mp_oracle.c`` compiled into a temporary
directory; the committed oracle is never modified. A mutant "survives" if every
pin still passes -- that would mean the pins cannot tell it from the real oracle.
"""
import os
import subprocess

import pytest

import oracle
import pins

MUTANTS = {
    "sample_std": ("v / (double)m", "v / (double)(m - 1)"),
    "no_mean_y": ("(y[k] - my) / sy", "y[k] / sy"),
    "windows_cross_segments": ("offs[s + 1] - offs[s]", "offs[nseg] - offs[s]"),
    "ties_to_highest": ("if (d < seg_best)", "if (d <= seg_best)"),
    "sign_flip": ("const double d = zx - zy;", "const double d = zx + zy;"),
    "index_off_by_one": ("seg_g = g;", "seg_g = g + 1;"),
    "no_elementwise_min": ("if (seg_best < best)", "if (1)"),
    "constant_never_detected": ("            return 0;\n    return 1;", "            return 0;\n    return 0;"),
    "constant_mixed_zero": ("    if (cx || cy)\n        return sqrt((double)m);", "    if (cx || cy)\n        return 0.0;"),
    "constant_both_sqrt_m": ("    if (cx && cy)\n        return 0.0;", "    if (cx && cy)\n        return sqrt((double)m);"),
    "mean_over_m_minus_1": ("const double mu = s / (double)m;", "const double mu = s / (double)(m - 1);"),
    "squared_distance": ("    return sqrt(acc);\n}", "    return acc;\n}"),
    "exclusion_asymmetric": ("if (g > i - excl && g < i + excl)", "if (g > i - excl && g <= i + excl)"),
    "exclusion_ignored": ("if (g > i - excl && g < i + excl)", "if (0)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = tmp_path / "mp_oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    oracle.build(force=True, src=str(mutated), out=str(so))
    lib = oracle.load(str(so))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            with __import__("numpy").errstate(all="ignore"):
                pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"mutant {name} passed every pin"
