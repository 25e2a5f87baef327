"""Tensor-core join (tcgen05: split BF16, TF32, single BF16) against the CPU oracle (needs a GB300).

Tolerance of both forms (the tensor-core contract): distances within 1e-3
absolute, indices exact where the oracle's best and second-best distances
differ by more than 1e-3. The finalisation recomputes the chosen pair's
distance exactly, and the kernels record every chunk whose approximate score
lies within twice the products' error bound of the best (TF32: 11-bit
operands; split BF16: 3 * 2^-18; single BF16: 8-bit operands; plus the FP32
sum), which the finalisation re-scores exactly. So the pick does not depend
on the products' rounding, for any form and window length.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import parity
import synthetic

pytestmark = pytest.mark.gpu

VARIANTS = {"bf16x3": 2, "tf32": 3, "bf16": 4}


@pytest.fixture(scope="module")
def ctxs(mp):
    cs = {name: mp.mp_init(device=0, kernel=k) for name, k in VARIANTS.items()}
    yield cs
    for c in cs.values():
        mp.mp_shutdown(c)


def check(variant, dist, idx, q, b, offs, m, rows=None, oracle_out=None):
    return parity.check(dist, idx, q, b, offs, m, rows=rows, atol=1e-3, oracle_out=oracle_out)


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
          # short windows whose spread is near the noise floor: the operands'
          # shifts multiply the TF32 rounding, and the width grows with them
          ("tf32", 16), ("tf32", 48), ("tf32", 128), ("tf32", 256),
          # one BF16 product: 8-bit operands, a wide width, many chunks re-scored
          ("bf16", 16), ("bf16", 128), ("bf16", 256)]


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
    for variant in ("tf32", "bf16x3", "bf16"):
        dist, idx = join(mp, ctxs[variant], w.query, w.dict_samples, w.offsets, w.m)
        rows = np.random.default_rng(3).choice(len(dist), 128, replace=False)
        check(variant, dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows)


def test_tc_matches_plain_on_random_walk_offsets(mp, ctxs):
    """Large offsets (random walk) exercise the shifts of the Hankel operands."""
    q = (synthetic.random_walk(5000, 31) + 3000.0).astype(np.float32)
    b = (synthetic.random_walk(6000, 32) - 2000.0).astype(np.float32)
    offs = np.array([0, 2500, 6000])
    for variant in ("tf32", "bf16x3", "bf16"):
        dist, idx = join(mp, ctxs[variant], q, b, offs, 128)
        check(variant, dist, idx, q, b, offs, 128, rows=np.arange(0, len(q) - 127, 7))


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_tc_near_ties_all_rows(mp, ctxs, variant):
    """ECG requests of the serving mix whose best and second-best windows lie about 1e-4 apart: within the
    TF32 products' error, so the pick rests on the near-tie records and the exact re-scoring."""
    for k in (0, 2):
        b, offs, q, m = _serving_mix_request(k)
        dist, idx = join(mp, ctxs[variant], q, b, offs, m)
        od, oi, od2 = oracle.ab_join(q, b, offs, m)
        assert int(((od2 - od) < 2e-4).sum()) >= 5, "the case must contain near ties"
        check(variant, dist, idx, q, b, offs, m, oracle_out=(od, oi, od2))


def _serving_mix_request(k):
    dicts = synthetic.serving_dictionaries(n_dicts=4, seed=100, min_log2=12, max_log2=14)
    rng = np.random.default_rng(0)
    for j in range(k + 1):
        n = int(2 ** rng.uniform(10, 14))
        m = int(rng.choice([64, 128, 256]))
        di = int(rng.integers(0, len(dicts)))
    src = synthetic.random_walk if k % 2 else synthetic.ecg_like
    b, offs = dicts[di]
    return b, offs, src(n, 1000 + k).astype(np.float32), m
