"""Autotuner, e_max (Sec. 3.3) and discords on the GPU join (needs a GB300)."""
from __future__ import annotations

import json

import numpy as np
import pytest

import oracle
import parity
import synthetic

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_persists_a_plain_grouping(mp, tmp_path):
    cache = tmp_path / "tune.jsonl"
    w = synthetic.workload("ecg_1m_m256", scale=1 / 8)
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_AUTO, tune_cache=str(cache))
    try:
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        kern, groups, ms = mp.mp_autotune(ctx, d, w.m, len(w.query), 1e-4)
        assert kern == mp.MP_KERNEL_PLAIN and groups >= 1 and ms > 0
        # a looser tolerance may admit split-BF16, but only forms that meet it
        kern3, _, _ = mp.mp_autotune(ctx, d, w.m, len(w.query), 1e-3)
        assert kern3 in (mp.MP_KERNEL_PLAIN, mp.MP_KERNEL_TC_BF16X3)
        lines = [json.loads(x) for x in cache.read_text().splitlines()]
        assert len(lines) == 2 and lines[0]["m"] == w.m and lines[0]["kernel"] == kern
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
    # a new context reloads the cache; AUTO joins of that shape use the choice
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_AUTO, tune_cache=str(cache))
    try:
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        dist, idx = mp.mp_ab_join(ctx, d, w.query, w.m)
        rows = np.random.default_rng(5).choice(len(dist), 96, replace=False)
        parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows,
                     atol=1e-4 if kern3 == mp.MP_KERNEL_PLAIN else 1e-3)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_emax_and_lemmas_on_gpu_joins(mp):
    """e_max from its definition and Lemma 1 / Lemma 2 for a dictionary cut from T_B."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 64
        tb = synthetic.ecg_like(8000, 41).astype(np.float32)
        ta = synthetic.ecg_like(3000, 42, n_malformed=4).astype(np.float32)
        db, offs = synthetic.cut_dictionary(tb, 16, 220)
        d = mp.mp_dict_load(ctx, db, offs, [m])
        e_max, arg = mp.mp_emax(ctx, d, tb, m)
        od, _, _ = oracle.ab_join(tb, db, offs, m)
        assert abs(e_max - od.max()) <= 1e-4
        assert abs(od[arg] - od.max()) <= 1e-4
        full = mp.mp_dict_load(ctx, tb, np.array([0, len(tb)]), [m])
        P, _ = mp.mp_ab_join(ctx, full, ta, m)
        Ph, _ = mp.mp_ab_join(ctx, d, ta, m)
        tol = 2e-4
        assert np.all(Ph >= P - tol), "Lemma 1 (no false negatives)"
        assert np.all(Ph - P <= e_max + tol), "Lemma 2 (max error)"
        mp.mp_dict_free(ctx, d)
        mp.mp_dict_free(ctx, full)
    finally:
        mp.mp_shutdown(ctx)


def test_discords_find_planted_malformed_beats(mp):
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 180
        train = synthetic.ecg_like(1 << 16, 51).astype(np.float32)  # normal beats only
        db, offs = synthetic.cut_dictionary(train, 32, 1024)
        q, (starts, malformed) = synthetic.ecg_like(1 << 15, 52, n_malformed=6, return_beats=True)
        q = q.astype(np.float32)
        d = mp.mp_dict_load(ctx, db, offs, [m])
        prof, _ = mp.mp_ab_join(ctx, d, q, m)
        e_max, _ = mp.mp_emax(ctx, d, train, m)
        idx, val, _ = mp.mp_top_discords(prof, 6, m // 2, e_max)
        bad = starts[malformed]
        # every top discord window overlaps a planted malformed beat
        hit = [np.any((bad < i + m) & (bad + 200 > i)) for i in idx]
        assert all(hit), (idx, bad)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
