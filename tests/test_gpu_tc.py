"""Tensor-core join (tcgen05, TF32 and split BF16) against the CPU oracle (needs a GB300).

Tolerance of the split-BF16 form: distances within 1e-3 absolute, indices
exact where the oracle's best and second-best distances differ by more than
1e-3 (the finalisation recomputes the chosen pair's distance exactly, so only
near-ties can move a distance).

The single-TF32 form rounds each operand to 11 significant bits, so its
correlation carries an error up to about 2 * 2^-11 * K (K >= 1 depends on the
shifts) and d^2 = 2m(1 - rho) up to 4m * 2^-11 * K; near-ties within that are
not resolved. Its checks: every reported distance is the exact distance of a
valid window (never below the oracle's minimum) and d^2 exceeds the oracle's
by at most 4m * 2^-10 (K <= 2 here); the index is exact where the oracle's
best and second-best d^2 differ by more than twice that.
"""
from __future__ import annotations

import numpy as np
import pytest

import parity
import synthetic

pytestmark = pytest.mark.gpu

VARIANTS = {"bf16x3": 2, "tf32": 3}


@pytest.fixture(scope="module")
def ctxs(mp):
    cs = {name: mp.mp_init(device=0, kernel=k) for name, k in VARIANTS.items()}
    yield cs
    for c in cs.values():
        mp.mp_shutdown(c)


def tf32_d2_tol(m):
    return 4.0 * m * 2.0**-10


def check(variant, dist, idx, q, b, offs, m, rows=None):
    if variant == "tf32":
        return parity.check_lower_precision(dist, idx, q, b, offs, m, tf32_d2_tol(m), rows=rows)
    return parity.check(dist, idx, q, b, offs, m, rows=rows, atol=1e-3)


def join(mp, ctx, q, b, offs, m):
    d = mp.mp_dict_load(ctx, b, offs, [m])
    try:
        return mp.mp_ab_join(ctx, d, q, m)
    finally:
        mp.mp_dict_free(ctx, d)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_tc_tiny(mp, ctxs, variant):
    # one CTA row block, tiles narrower than 256 and one window past a tile edge
    q = synthetic.random_walk(200, 5).astype(np.float32)
    b = synthetic.random_walk(700, 6).astype(np.float32)
    offs = np.array([0, 300, 700])
    dist, idx = join(mp, ctxs[variant], q, b, offs, 64)
    check(variant, dist, idx, q, b, offs, 64)


SHAPES = [("bf16x3", 16), ("bf16x3", 48), ("bf16x3", 128), ("bf16x3", 256),
          # single TF32 is not used below m = 48: for short windows whose spread is
          # near the noise floor the shift of the operands multiplies its error
          ("tf32", 48), ("tf32", 128), ("tf32", 256)]


@pytest.mark.parametrize("variant,m", SHAPES)
def test_tc_small_shapes(mp, ctxs, variant, m):
    q = synthetic.ecg_like(1500, 7 + m).astype(np.float32)
    lens = [m - 1, 2 * m + 37, 500, 1300, m]
    b = synthetic.ecg_like(sum(lens), 8 + m).astype(np.float32)
    offs = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
    dist, idx = join(mp, ctxs[variant], q, b, offs, m)
    check(variant, dist, idx, q, b, offs, m)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_tc_ecg_m256_all_rows(mp, ctxs, variant):
    w = synthetic.workload("ecg_1m_m256", scale=1 / 128)
    dist, idx = join(mp, ctxs[variant], w.query, w.dict_samples, w.offsets, w.m)
    check(variant, dist, idx, w.query, w.dict_samples, w.offsets, w.m)


def test_tc_transport_m512_sampled(mp, ctxs):
    w = synthetic.workload("transport_4m_m512", scale=1 / 16)
    for variant in ("tf32", "bf16x3"):
        dist, idx = join(mp, ctxs[variant], w.query, w.dict_samples, w.offsets, w.m)
        rows = np.random.default_rng(3).choice(len(dist), 128, replace=False)
        check(variant, dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows)


def test_tc_matches_plain_on_random_walk_offsets(mp, ctxs):
    """Large offsets (random walk) exercise the shifts of the Hankel operands."""
    q = (synthetic.random_walk(5000, 31) + 3000.0).astype(np.float32)
    b = (synthetic.random_walk(6000, 32) - 2000.0).astype(np.float32)
    offs = np.array([0, 2500, 6000])
    for variant in ("tf32", "bf16x3"):
        dist, idx = join(mp, ctxs[variant], q, b, offs, 128)
        check(variant, dist, idx, q, b, offs, 128, rows=np.arange(0, len(q) - 127, 7))
