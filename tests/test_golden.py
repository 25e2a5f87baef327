"""Oracle distances against the hand-derived values in tests/golden/closed_forms.txt."""
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def load_cases():
    cases = []
    with open(os.path.join(HERE, "golden", "closed_forms.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            x, y, d, _why = [p.strip() for p in line.split(";", 3)]
            cases.append((np.array(x.split(), float), np.array(y.split(), float), float(d)))
    return cases


def test_golden_closed_forms(oracle_lib):
    cases = load_cases()
    assert len(cases) >= 7
    for x, y, d in cases:
        got = oracle.pair_distance(x, y, lib=oracle_lib)
        assert abs(got - d) <= 1e-12, (x, y, got, d)
