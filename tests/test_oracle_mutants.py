"""Plant plausible mistakes in copies of the oracle and check that the pins catch each.

Each mutant is a textual edit of ``oracle/mp_oracle.c`` compiled into a temporary
directory, or of ``oracle/__init__.py`` run as a fresh module; the committed
oracle is never modified. A mutant "survives" if every
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


# Mistakes planted in the Python half of the oracle (Algorithm 1 and the
# correlation output). The edited source runs as a fresh module with the
# original's file path (so that it finds the compiled C part), and the pins
# use it in place of the committed module for the duration of the test.
PY_MUTANTS = {
    "learn_takes_argmax": ("j = int(np.argmin(np.where(finite, Pp, np.inf)))",
                           "j = int(np.argmax(np.where(finite, Pp, -np.inf)))"),
    "learn_excludes_one_window": ("excluded[max(0, j - half):min(nq, j + half)] = True", "excluded[j] = True"),
    "learn_folds_with_max": ("S = Sp if it == 0 else np.minimum(S, Sp)", "S = Sp if it == 0 else np.maximum(S, Sp)"),
    "learn_context_doubled": ("pad = int(np.floor((k_context - 1.0) * m / 2.0))",
                              "pad = int(np.floor((k_context - 1.0) * m))"),
    "corr_scale_m": ("1.0 - d * d / (2.0 * m)", "1.0 - d * d / m"),
}


def _pins_failed_by(src, monkeypatch):
    import types

    import numpy as np

    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = oracle.__file__
    exec(compile(src, oracle.__file__, "exec"), mod.__dict__)
    monkeypatch.setattr(pins, "oracle", mod)
    lib = oracle.load()
    caught = []
    for pin in pins.ALL_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    return caught


def test_python_oracle_loaded_this_way_passes_every_pin(monkeypatch):
    # the control for the mutants below: the unedited source, run as a fresh module
    assert _pins_failed_by(open(oracle.__file__).read(), monkeypatch) == []


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_mutant_is_caught(name, monkeypatch):
    old, new = PY_MUTANTS[name]
    src = open(oracle.__file__).read()
    assert src.count(old) == 1, f"mutation site for {name} not found"
    assert _pins_failed_by(src.replace(old, new), monkeypatch), f"mutant {name} passed every pin"
