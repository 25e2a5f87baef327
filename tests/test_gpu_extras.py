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
        # every form picks exactly, so any may win; the choice records the tolerance
        kern3, _, _ = mp.mp_autotune(ctx, d, w.m, len(w.query), 1e-3)
        assert kern3 in (mp.MP_KERNEL_PLAIN, mp.MP_KERNEL_TC_BF16X3, mp.MP_KERNEL_TC_TF32, mp.MP_KERNEL_TC_BF16)
        lines = [json.loads(x) for x in cache.read_text().splitlines()]
        assert len(lines) == 2 and lines[0]["m"] == w.m and lines[0]["kernel"] == kern
        assert lines[0]["tolerance"] == 1e-4 and lines[1]["tolerance"] == 1e-3
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
    # a new context reloads the cache; AUTO joins of that shape use the choice
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_AUTO, tune_cache=str(cache))
    try:
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        assert mp.mp_plan_join(ctx, d, mp.MP_F32, len(w.query), w.m)["kernel"] == kern3
        dist, idx = mp.mp_ab_join(ctx, d, w.query, w.m)
        rows = np.random.default_rng(5).choice(len(dist), 96, replace=False)
        parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows, atol=1e-4)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_plan_join(mp):
    w = synthetic.workload("ecg_1m_m256", scale=1 / 8)
    ctx = mp.mp_init(device=0)
    try:
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        p = mp.mp_plan_join(ctx, d, mp.MP_F32, len(w.query), w.m)
        assert p["kernel"] == mp.MP_KERNEL_PLAIN and p["tc_seeds"] == 1 and p["row_chunks"] >= 1
        # a span is one segment's run of windows in one group: each segment gives at least one, and
        # each segment boundary inside a group adds one to the groups
        n_seg = len(w.offsets) - 1
        assert n_seg <= p["spans"] <= p["column_groups"] + n_seg - 1
        assert p["workspace_bytes"] > 0
        mp.mp_set_kernel(ctx, mp.MP_KERNEL_TC_BF16)
        p1 = mp.mp_plan_join(ctx, d, mp.MP_F32, len(w.query), w.m)
        assert p1["kernel"] == mp.MP_KERNEL_TC_BF16 and p1["tc_seeds"] == 0
        assert p1["workspace_bytes"] == p["workspace_bytes"]  # reserved for every form
        with pytest.raises(mp.MPError):
            mp.mp_plan_join(ctx, d, mp.MP_F32, len(w.query), 3)
        with pytest.raises(mp.MPError):
            mp.mp_plan_join(ctx, d, mp.MP_F64, len(w.query), w.m)  # the dictionary holds float32
        mp.mp_dict_free(ctx, d)
        # FP64: the plain form, no tensor-core seeds
        d64 = mp.mp_dict_load(ctx, w.dict_samples.astype(np.float64), w.offsets, [w.m])
        p2 = mp.mp_plan_join(ctx, d64, mp.MP_F64, 4096, w.m)
        assert p2["kernel"] == mp.MP_KERNEL_PLAIN and p2["tc_seeds"] == 0
        mp.mp_dict_free(ctx, d64)
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


def test_correlation_output_matches_oracle(mp):
    """mp_ab_join_corr: the largest rho = 1 - d^2/(2m) per row and the join's index (Sec. 2.1)."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 96
        q = synthetic.ecg_like(6000, 61, n_malformed=3).astype(np.float32)
        b = synthetic.ecg_like(9000, 62).astype(np.float32)
        b[4000:4200] = 1.5  # constant dictionary windows
        offs = np.array([0, 2500, 2700, 6000, 9000])
        d = mp.mp_dict_load(ctx, b, offs, [m])
        rho, idx = mp.mp_ab_join_corr(ctx, d, q, m)
        dist, idx2 = mp.mp_ab_join(ctx, d, q, m)
        assert np.array_equal(idx, idx2)
        np.testing.assert_allclose(rho, 1.0 - dist ** 2 / (2 * m), rtol=0, atol=1e-12)
        orho, oidx = oracle.ab_join_corr(q, b, offs, m)
        # the distance tolerance 1e-4 near d carries to rho as d * 1e-4 / m
        tol = 1e-4 * np.maximum(dist, 1.0) / m
        assert np.all(np.abs(rho - orho) <= tol + 1e-9)
        assert np.all((rho <= 1.0 + 1e-9) & (rho >= -1.0 - 1e-9))
        mp.mp_dict_free(ctx, d)
        # no dictionary window at all: -inf / -1
        d = mp.mp_dict_load(ctx, b[:90], np.array([0, 90]), [m])
        rho, idx = mp.mp_ab_join_corr(ctx, d, q[:500], m)
        assert np.all(np.isneginf(rho)) and np.all(idx == -1)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_stream_submit_equals_one_shot_join(mp):
    """Appends without waiting (each one a serving request, batched with the others) give the one-shot join."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 128
        train = synthetic.ecg_like(1 << 15, 73).astype(np.float32)
        db, offs = synthetic.cut_dictionary(train, 16, 700)
        d = mp.mp_dict_load(ctx, db, offs, [m])
        x = synthetic.ecg_like(30000, 74, n_malformed=4).astype(np.float32)
        full_d, full_i = mp.mp_ab_join(ctx, d, x, m)
        st = mp.mp_stream_open(ctx, d, mp.MP_F32, m)
        cuts = [0, 100, 127, 1024, 2048, 3000, 4096, 9000, 20000, 29000, 30000]
        pieces = []
        for a, c in zip(cuts[:-1], cuts[1:]):
            od, oi = np.full(c - a, np.nan), np.full(c - a, -7, dtype=np.int64)
            t, k, first = mp.mp_stream_submit(st, x[a:c], od, oi)
            assert k == max(0, c - m + 1) - max(0, a - m + 1) and (t != 0) == (k > 0)
            pieces.append((t, od, oi, k, first))
        for t, *_ in pieces:
            if t:
                while mp.mp_poll(ctx, t)[0] == mp.MP_PENDING:
                    pass
        mp.mp_stream_close(st)
        got_d = np.concatenate([od[:k] for _, od, _, k, _ in pieces])
        got_i = np.concatenate([oi[:k] for _, _, oi, k, _ in pieces])
        assert [f for t, *_, f in pieces if t][0] == 0 and len(got_d) == len(full_d)
        np.testing.assert_allclose(got_d, full_d, rtol=0, atol=1e-4)
        diff = got_i != full_i  # a different pick only between windows the re-scoring cannot tell apart
        assert diff.mean() < 1e-3 and np.all(np.abs(got_d[diff] - full_d[diff]) <= 1e-4)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_streaming_join_equals_one_shot_join(mp):
    """Appending a series in uneven pieces joins every window once, as the one-shot join does."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 128
        train = synthetic.ecg_like(1 << 15, 71).astype(np.float32)
        db, offs = synthetic.cut_dictionary(train, 16, 700)
        d = mp.mp_dict_load(ctx, db, offs, [m])
        x = synthetic.ecg_like(20000, 72, n_malformed=4).astype(np.float32)
        full_d, full_i = mp.mp_ab_join(ctx, d, x, m)
        st = mp.mp_stream_open(ctx, d, mp.MP_F32, m)
        cuts = [0, 50, 127, 128, 900, 901, 5000, 12000, 19999, 20000]
        got_d, got_i, firsts = [], [], []
        for a, c in zip(cuts[:-1], cuts[1:]):
            sd, si, first = mp.mp_stream_append(st, x[a:c])
            assert len(sd) == max(0, c - m + 1) - max(0, a - m + 1)
            if len(sd):
                firsts.append(first)
            got_d.append(sd)
            got_i.append(si)
        # an empty append changes nothing
        sd, si, first = mp.mp_stream_append(st, x[:0])
        assert len(sd) == 0 and first == len(x) - m + 1
        mp.mp_stream_close(st)
        got_d = np.concatenate(got_d)
        got_i = np.concatenate(got_i)
        assert len(got_d) == len(full_d) and firsts[0] == 0
        np.testing.assert_allclose(got_d, full_d, rtol=0, atol=1e-4)
        diff = got_i != full_i
        assert diff.mean() < 1e-3 and np.all(np.abs(got_d[diff] - full_d[diff]) <= 1e-4)
        rows = np.random.default_rng(3).choice(len(got_d), 64, replace=False)
        parity.check(got_d, got_i, x, db, offs, m, rows=rows, atol=1e-4)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_self_join_matches_oracle(mp):
    """mp_self_join (Algorithm 1's P_B) against the oracle's self-join, constant windows included."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 64
        x = synthetic.random_walk(5000, 91).astype(np.float32)
        x[2000:2200] = x[2000]      # a constant run: windows inside it are constant
        x[3500:3580] = -4.0         # a second one, farther than the exclusion zone
        excl = (m + 1) // 2
        d, i = mp.mp_self_join(ctx, x, m, excl)
        od, oi = oracle.self_join(x, m, excl)
        assert np.all(np.abs(d - od) <= 1e-4)
        g = np.arange(len(d))
        assert np.all((i < 0) | (np.abs(i - g) >= excl)), "a trivial match was reported"
        # where the oracle's pick is clearly best, the index must match
        rows = np.random.default_rng(1).choice(len(d), 300, replace=False)
        for r in rows:
            if i[r] != oi[r]:
                dg = oracle.pair_distance(x[r : r + m], x[i[r] : i[r] + m])
                assert dg <= od[r] + 1e-4
        # constant windows: 0 to another constant window outside the zone
        cst = np.arange(2000, 2200 - m + 1)
        assert np.all(d[cst] == 0.0) and np.all(np.abs(i[cst] - cst) >= excl)
    finally:
        mp.mp_shutdown(ctx)


def test_learn_dictionary_matches_oracle(mp):
    """Algorithm 1 on the GPU picks the same windows as the oracle and keeps its error bound."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        m = 64
        x = synthetic.ecg_like(12000, 93).astype(np.float32)
        segs, chosen, bound = mp.mp_learn_dictionary(ctx, x, m, 1.5, mp.MP_LEARN_MEMORY, 2000)
        osegs, ochosen, obound = oracle.learn_dictionary(x, m, 1.5, "memory", 2000)
        assert chosen == ochosen and segs == osegs
        assert abs(bound - obound) <= 1e-3
        # the learned dictionary's e_max (by the GPU join) is within the bound
        samples = np.concatenate([x[a : a + L] for a, L in segs])
        offs = np.concatenate(([0], np.cumsum([L for _, L in segs])))
        d = mp.mp_dict_load(ctx, samples, offs, [m])
        e_max, _ = mp.mp_emax(ctx, d, x, m)
        assert e_max <= bound + 1e-3
        mp.mp_dict_free(ctx, d)
        # the e_max terminal condition
        segs2, chosen2, bound2 = mp.mp_learn_dictionary(ctx, x, m, 1.5, mp.MP_LEARN_EMAX, bound)
        assert bound2 <= bound + 1e-6 and chosen2 == chosen[: len(chosen2)]
    finally:
        mp.mp_shutdown(ctx)


def test_repeated_small_joins_replay_a_graph(mp):
    """A synchronous join repeated with the same shape runs, from its second call on, as one captured CUDA graph.
    Every call gives the first call's results bit for bit; a query with NaN at that shape is still refused with
    the outputs untouched; after its dictionary is freed, a new dictionary of the same shape gets its own
    results (the cached graph held the old one's pointers)."""
    w = synthetic.workload("ecg_1m_m256", scale=1 / 256)
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        ref_d, ref_i = mp.mp_ab_join(ctx, d, w.query, w.m)
        for _ in range(4):
            dist, idx = mp.mp_ab_join(ctx, d, w.query, w.m)
            assert np.array_equal(dist, ref_d) and np.array_equal(idx, ref_i)
        # another query of the same length through the cached graph
        q2 = synthetic.ecg_like(len(w.query), 77).astype(np.float32)
        d2, i2 = mp.mp_ab_join(ctx, d, q2, w.m)
        rows = np.arange(0, len(d2), 53)
        parity.check(d2, i2, q2, w.dict_samples, w.offsets, w.m, rows=rows, atol=1e-4)
        # NaN at a cached shape: refused, nothing written
        bad = w.query.copy()
        bad[len(bad) // 2] = np.nan
        out_d = np.full(len(ref_d), -5.0)
        out_i = np.full(len(ref_d), -9, dtype=np.int64)
        with pytest.raises(mp.MPError) as e:
            mp._check(mp.lib.mp_ab_join(ctx, d, mp._ptr(bad), mp.MP_F32, len(bad), w.m, mp._ptr(out_d),
                                        mp._ptr(out_i)))
        assert e.value.code == mp.MP_E_ARG
        assert np.all(out_d == -5.0) and np.all(out_i == -9)
        mp.mp_dict_free(ctx, d)
        # a different dictionary of the same shape
        b2 = synthetic.ecg_like(len(w.dict_samples), 78).astype(np.float32)
        dn = mp.mp_dict_load(ctx, b2, w.offsets, [w.m])
        for _ in range(3):
            d3, i3 = mp.mp_ab_join(ctx, dn, w.query, w.m)
        parity.check(d3, i3, w.query, b2, w.offsets, w.m, rows=rows, atol=1e-4)
        mp.mp_dict_free(ctx, dn)
    finally:
        mp.mp_shutdown(ctx)
