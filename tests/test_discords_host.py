"""Discord extraction and certification (host code of the library, CPU only)."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as g

    g._load_build_module().build()
    import paper_2112_12965_gb300 as lib

    return lib


def brute_top_discords(p, k, excl):
    p = np.asarray(p, dtype=float)
    blocked = np.zeros(len(p), bool)
    out = []
    for _ in range(k):
        cand = np.where(~blocked & np.isfinite(p), p, -np.inf)
        if not np.isfinite(cand).any():
            break
        b = int(np.argmax(cand))  # first index among equal maxima
        out.append((b, p[b]))
        blocked[max(0, b - excl): b + excl + 1] = True
    return out


def test_top_discords_match_brute_force(mp):
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(1, 400))
        p = rng.random(n) * 10
        p[rng.random(n) < 0.05] = np.inf  # windows without a neighbour are skipped
        k = int(rng.integers(0, 12))
        excl = int(rng.integers(0, 30))
        idx, val, _ = mp.mp_top_discords(p, k, excl)
        ref = brute_top_discords(p, k, excl)
        assert list(idx) == [r[0] for r in ref]
        assert np.array_equal(val, [r[1] for r in ref])


def test_top1_certificate_follows_guarantee_2(mp):
    p = np.array([1.0, 1.2, 5.0, 1.1, 1.0, 3.9, 1.0])
    # lead of 5.0 over the best value outside +-1 of index 2 (3.9) is 1.1
    _, _, cert = mp.mp_top_discords(p, 1, 1, e_max=1.0)
    assert cert
    _, _, cert = mp.mp_top_discords(p, 1, 1, e_max=1.2)
    assert not cert
    # a huge exclusion zone leaves no competitor: certified for any finite e_max
    _, _, cert = mp.mp_top_discords(p, 1, 10, e_max=100.0)
    assert cert
