"""GPU join through the C ABI against the CPU oracle (needs a GB300)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import parity
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(mp):
    c = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    yield c
    mp.mp_shutdown(c)


def join(mp, ctx, q, b, offs, m, ms=None):
    d = mp.mp_dict_load(ctx, b, offs, [m] if ms is None else ms)
    try:
        return mp.mp_ab_join(ctx, d, q, m)
    finally:
        mp.mp_dict_free(ctx, d)


def test_window_stats_match_oracle(mp, ctx):
    import torch

    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(3000).cumsum() + 5000.0, np.full(300, 7.25),
                        rng.standard_normal(700)]).astype(np.float32)
    for m in (4, 64, 257, 1024):
        xt = torch.from_numpy(x).cuda()
        nw = len(x) - m + 1
        mean = torch.empty(nw, dtype=torch.float64, device="cuda")
        inv = torch.empty_like(mean)
        cst = torch.empty(nw, dtype=torch.uint8, device="cuda")
        mp.mp_window_stats(ctx, xt.data_ptr(), mp.MP_F32, len(x), m, mean.data_ptr(), inv.data_ptr(), cst.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        om, osd, oc = oracle.window_stats(x, m)
        assert np.array_equal(cst.cpu().numpy().astype(bool), oc)
        np.testing.assert_allclose(mean.cpu().numpy(), om, rtol=1e-12, atol=1e-9)
        inv_o = np.where(oc, 0.0, 1.0 / np.where(oc, 1.0, osd))
        np.testing.assert_allclose(inv.cpu().numpy(), inv_o, rtol=1e-9)


def test_fp64_random_walk_all_rows(mp, ctx):
    w = synthetic.workload("rw_fp64_4k")
    dist, idx = join(mp, ctx, w.query, w.dict_samples, w.offsets, w.m)
    r = parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, atol=1e-8, gap=1e-6)
    assert r["n_rows"] == 4033


def test_fp32_ecg_all_rows_small(mp, ctx):
    w = synthetic.workload("ecg_1m_m256", scale=1 / 128)
    dist, idx = join(mp, ctx, w.query, w.dict_samples, w.offsets, w.m)
    parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, atol=1e-4)


def test_fp32_ecg_full_size_sampled_rows(mp, ctx):
    w = synthetic.workload("ecg_1m_m256")
    dist, idx = join(mp, ctx, w.query, w.dict_samples, w.offsets, w.m)
    assert len(dist) == 1048321
    # 2^14 random rows (about 20 s of the oracle on the host's cores), both ends, and the 64 farthest rows
    # (the planted malformed beats)
    rows = _sampled_rows(dist, 1 << 14, 0, n_top=64, n_ends=64)
    parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows, atol=1e-4)
    # properties that hold at any size
    assert np.all((dist >= 0) & (dist <= 2 * math.sqrt(w.m) + 1e-9))
    assert np.all((idx >= 0) & (idx < len(w.dict_samples)))


def _sampled_rows(dist, n_random, seed, n_top=0, n_ends=16):
    """Random rows, the first and last rows, and the rows of the n_top largest distances."""
    rng = np.random.default_rng(seed)
    parts = [rng.choice(len(dist), n_random, replace=False), np.arange(0, n_ends),
             np.arange(len(dist) - n_ends, len(dist))]
    if n_top:
        parts.append(np.argsort(dist)[-n_top:])
    return np.unique(np.concatenate(parts))


def test_transport_m512_full_size_sampled_rows(mp, ctx):
    """Transportation-like query of 2^22 samples against 256 x 2048 segments, m = 512, at full size."""
    w = synthetic.workload("transport_4m_m512")
    dist, idx = join(mp, ctx, w.query, w.dict_samples, w.offsets, w.m)
    assert len(dist) == (1 << 22) - 512 + 1
    rows = _sampled_rows(dist, 2048, 1, n_top=32)
    parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows, atol=1e-4)
    assert np.all((dist >= 0) & (dist <= 2 * math.sqrt(w.m) + 1e-9))


def test_ecg_m1024_dictionary_full_size_sampled_rows(mp, ctx):
    """ECG-like query of 2^24 samples (200 planted malformed beats) against 128 x 2048 segments cut from a
    normal-beat training series, m = 1024, at full size. Windows longer than 512 take the per-pass
    finalisation, and the top-seed matrix (17 GB at once) is built in row chunks. The rows of the 256 largest
    distances lie on planted beats."""
    w = synthetic.workload("ecg_16m_m1024_dict")
    dist, idx = join(mp, ctx, w.query, w.dict_samples, w.offsets, w.m)
    assert len(dist) == (1 << 24) - 1024 + 1
    rows = _sampled_rows(dist, 1024, 2, n_top=256, n_ends=8)
    parity.check(dist, idx, w.query, w.dict_samples, w.offsets, w.m, rows=rows, atol=1e-4)
    assert np.all((dist >= 0) & (dist <= 2 * math.sqrt(w.m) + 1e-9))


def test_ecg_m1024_original_series_and_lemma_1(mp, ctx):
    """A quarter-size query (2^22 samples) against the whole training series as one segment (2^20 samples,
    m = 1024): sampled rows against the oracle, and Lemma 1 (the join against the dictionary cut from that
    series never undercuts the join against the series) on every row."""
    wo = synthetic.workload("ecg_16m_m1024_orig", scale=0.25)
    wd = synthetic.workload("ecg_16m_m1024_dict", scale=0.25)
    p_orig, i_orig = join(mp, ctx, wo.query, wo.dict_samples, wo.offsets, wo.m)
    p_dict, _ = join(mp, ctx, wd.query, wd.dict_samples, wd.offsets, wd.m)
    rows = _sampled_rows(p_orig, 16, 3, n_top=4, n_ends=2)
    parity.check(p_orig, i_orig, wo.query, wo.dict_samples, wo.offsets, wo.m, rows=rows, atol=1e-4)
    assert np.all(p_dict >= p_orig - 1e-4)


EDGE_CASES = {
    # name: (query length, segment lengths, m, generator)
    "ragged_segments": (3001, [700, 129, 64, 1500, 63, 2], 64, "rw"),
    "m4": (400, [50, 3, 1, 4, 70], 4, "rw"),
    "m37_odd": (1777, [300, 36, 37, 38, 900], 37, "ecg"),
    "one_row": (100, [250, 300], 100, "rw"),
    "one_window_segments": (2500, [96] * 40, 96, "rw"),
    "many_tiny_segments": (5000, [20 + (k % 7) for k in range(300)], 16, "ecg"),
    "long_single_segment": (3000, [9000], 200, "ecg"),
    "rows_span_cta_tail": (2560 + 639 + 300, [2000, 1000], 300, "rw"),
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_edge_cases(mp, ctx, name):
    n, lens, m, gen = EDGE_CASES[name]
    rng_seed = sum(map(ord, name))
    src = synthetic.random_walk if gen == "rw" else synthetic.ecg_like
    q = src(n, rng_seed).astype(np.float32)
    b = src(int(sum(lens)), rng_seed + 1).astype(np.float32)
    offs = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
    dist, idx = join(mp, ctx, q, b, offs, m)
    parity.check(dist, idx, q, b, offs, m, atol=1e-4)


def test_no_dictionary_window(mp, ctx):
    q = synthetic.random_walk(500, 3).astype(np.float32)
    b = synthetic.random_walk(90, 4).astype(np.float32)
    dist, idx = join(mp, ctx, q, b, np.array([0, 30, 60, 90]), 31)
    assert np.all(np.isinf(dist)) and np.all(idx == -1)


def test_constant_windows(mp, ctx):
    rng = np.random.default_rng(9)
    q = np.concatenate([rng.standard_normal(300), np.full(100, 2.5), rng.standard_normal(300)]).astype(np.float32)
    b = np.concatenate([rng.standard_normal(400), np.full(80, -1.0), rng.standard_normal(400)]).astype(np.float32)
    offs = np.array([0, 350, 500, 880])
    for m in (16, 50):
        dist, idx = join(mp, ctx, q, b, offs, m)
        parity.check(dist, idx, q, b, offs, m, atol=1e-4)
    # no constant dictionary window: constant query rows are sqrt(m) from every window, lowest index wins
    b2 = rng.standard_normal(600).astype(np.float32)
    dist, idx = join(mp, ctx, q, b2, np.array([0, 600]), 16)
    crow = np.arange(300, 300 + 100 - 16 + 1)
    assert np.allclose(dist[crow], 4.0) and np.all(idx[crow] == 0)


def test_planted_copy_and_segment_junction(mp, ctx):
    rng = np.random.default_rng(11)
    m = 64
    b = rng.standard_normal(3000).cumsum().astype(np.float32)
    offs = np.array([0, 1000, 2000, 3000])
    q = rng.standard_normal(4000).cumsum().astype(np.float32)
    g = 1000 + 321
    q[1500 : 1500 + m] = b[g : g + m]
    j = 2000 - m // 2
    q[3000 : 3000 + m] = b[j : j + m]
    dist, idx = join(mp, ctx, q, b, offs, m)
    assert idx[1500] == g and dist[1500] < 1e-3
    assert idx[3000] != j and dist[3000] > 0.05
    d1, i1 = join(mp, ctx, q, b, np.array([0, 1000, 3000]), m)
    assert i1[3000] == j and d1[3000] < 1e-3


def test_device_api_matches_host_api_and_is_deterministic(mp, ctx):
    import torch

    w = synthetic.workload("ecg_1m_m256", scale=1 / 32)
    d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
    try:
        hd, hi = mp.mp_ab_join(ctx, d, w.query, w.m)
        hd2, hi2 = mp.mp_ab_join(ctx, d, w.query, w.m)
        assert np.array_equal(hd, hd2) and np.array_equal(hi, hi2)
        qt = torch.from_numpy(w.query).cuda()
        nq = len(w.query) - w.m + 1
        dd = torch.empty(nq, dtype=torch.float64, device="cuda")
        di = torch.empty(nq, dtype=torch.int64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            mp.mp_ab_join_device(ctx, d, qt.data_ptr(), mp.MP_F32, len(w.query), w.m, dd.data_ptr(), di.data_ptr(),
                                 s.cuda_stream)
        s.synchronize()
        assert np.array_equal(dd.cpu().numpy(), hd) and np.array_equal(di.cpu().numpy(), hi)
    finally:
        mp.mp_dict_free(ctx, d)


def test_argument_errors(mp, ctx):
    b = synthetic.random_walk(1000, 1).astype(np.float32)
    d = mp.mp_dict_load(ctx, b, [0, 1000], [32])
    try:
        q = synthetic.random_walk(200, 2).astype(np.float32)
        for bad_m in (1, 2, 3, 201, 8193):
            with pytest.raises(mp.MPError) as e:
                mp.mp_ab_join(ctx, d, q, bad_m)
            assert e.value.code == mp.MP_E_ARG
        qn = q.copy()
        qn[17] = np.nan
        with pytest.raises(mp.MPError) as e:
            mp.mp_ab_join(ctx, d, qn, 32)
        assert e.value.code == mp.MP_E_ARG
        # through the C call: the caller's outputs stay untouched, the context stays usable
        nq = len(qn) - 32 + 1
        od, oi = np.full(nq, 7.0), np.full(nq, 7, dtype=np.int64)
        rc = mp.lib.mp_ab_join(ctx, d, qn.ctypes.data, mp.MP_F32, len(qn), 32, od.ctypes.data, oi.ctypes.data)
        assert rc == mp.MP_E_ARG and np.all(od == 7.0) and np.all(oi == 7)
        dist, idx = mp.mp_ab_join(ctx, d, q, 32)
        assert np.all(idx >= 0) and np.all(np.isfinite(dist))
        with pytest.raises(mp.MPError) as e:
            mp.mp_ab_join(ctx, d, q.astype(np.float64), 32)
        assert e.value.code == mp.MP_E_ARG
        with pytest.raises(mp.MPError) as e:
            mp.mp_dict_load(ctx, b, [0, 600, 500, 1000])
        assert e.value.code == mp.MP_E_ARG
    finally:
        mp.mp_dict_free(ctx, d)


def test_profile_phases(mp, ctx):
    w = synthetic.workload("ecg_1m_m256", scale=1 / 16)
    d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
    try:
        mp.mp_profile(ctx, True)
        mp.mp_profile_read(ctx, reset=True)
        for _ in range(3):
            mp.mp_ab_join(ctx, d, w.query, w.m)
        ms, n = mp.mp_profile_read(ctx, reset=True)
        # stats, join, finalisation, and the FP32 plain join's tensor-core seeds (3.2e9 pairs)
        assert mp.mp_plan_join(ctx, d, mp.MP_F32, len(w.query), w.m)["tc_seeds"] == 1
        assert list(n) == [3, 3, 3, 3, 3] and np.all(ms > 0)
        # a join below 2^31 pairs computes its seeds in the plain kernel
        q = w.query[: 8192 + w.m - 1]
        assert mp.mp_plan_join(ctx, d, mp.MP_F32, len(q), w.m)["tc_seeds"] == 0
        for _ in range(3):
            mp.mp_ab_join(ctx, d, q, w.m)
        ms, n = mp.mp_profile_read(ctx, reset=True)
        assert list(n) == [3, 3, 3, 0, 0] and np.all(ms[:3] > 0)
    finally:
        mp.mp_profile(ctx, False)
        mp.mp_dict_free(ctx, d)


def _serving_mix_request(k):
    """Request k of the serving test's seeded mix: (dictionary samples, offsets, query, m)."""
    dicts = synthetic.serving_dictionaries(n_dicts=4, seed=100, min_log2=12, max_log2=14)
    rng = np.random.default_rng(0)
    for j in range(k + 1):
        n = int(2 ** rng.uniform(10, 14))
        m = int(rng.choice([64, 128, 256]))
        di = int(rng.integers(0, len(dicts)))
    src = synthetic.random_walk if k % 2 else synthetic.ecg_like
    b, offs = dicts[di]
    return b, offs, src(n, 1000 + k).astype(np.float32), m


@pytest.mark.parametrize("k", [0, 2])
def test_near_ties_all_rows(mp, ctx, k):
    """ECG queries with rows whose best and second-best windows are about 1e-4 apart.

    The FP32 recurrence's rounding (about 1e-6 in correlation) can misorder such
    windows; the plain kernel records near ties and the finalisation re-scores
    them exactly, so every row's distance must be within 1e-4 of the oracle's.
    """
    b, offs, q, m = _serving_mix_request(k)
    dist, idx = join(mp, ctx, q, b, offs, m)
    od, oi, od2 = oracle.ab_join(q, b, offs, m)
    assert int(((od2 - od) < 2e-4).sum()) >= 5, "the case must contain near ties"
    parity.check(dist, idx, q, b, offs, m, atol=1e-4, oracle_out=(od, oi, od2))


def test_repeated_segments_rescore_every_tied_chunk(mp, ctx):
    """A dictionary of 16 exact copies of one segment: each row's best window
    ties in every copy, so the column groups hand the finalisation many
    near-tie candidates per row (more than it keeps per window in shared
    memory, which sends it back to the records). Every row's distance must
    still match the oracle's, and the chosen window must be at that distance.
    """
    m = 64
    seg = synthetic.ecg_like(301, 91).astype(np.float32)
    b = np.tile(seg, 16)
    offs = (np.arange(17) * 301).astype(np.int64)
    q = synthetic.ecg_like(3000, 92).astype(np.float32)
    dist, idx = join(mp, ctx, q, b, offs, m)
    od, oi, od2 = oracle.ab_join(q, b, offs, m)
    assert np.all(od2 - od < 1e-9), "every best window must tie with its copies"
    parity.check(dist, idx, q, b, offs, m, atol=1e-4, oracle_out=(od, oi, od2))


def test_drifting_offset_series_all_rows(mp, ctx):
    """Large offsets and drift: the seeds' centring must keep FP32 products small.

    m = 100 is no multiple of the tensor-core K step, the query has a ragged
    number of rows (not a multiple of the 640 rows a warp seeds), and the
    dictionary's segments have uneven lengths.
    """
    rng = np.random.default_rng(21)
    m = 100
    q = (rng.standard_normal(3 * 2048 + 777 + m - 1).cumsum() * 3.0 + 2.0e4).astype(np.float32)
    lens = [900, 101, 100, 2500, 333]
    b = (rng.standard_normal(sum(lens)).cumsum() * 5.0 - 3.0e4).astype(np.float32)
    offs = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
    dist, idx = join(mp, ctx, q, b, offs, m)
    parity.check(dist, idx, q, b, offs, m, atol=1e-4)


def test_large_join_runs_in_row_chunks(mp, ctx):
    """A join whose top-seed matrix would pass its 2 GiB cap runs in row chunks.

    A dictionary of 2^20 samples makes each seed row about 4 MB, so a chunk is
    512 seed rows of 640 query windows = 327,680 query windows, and a query of
    700,000 windows runs in three chunks. Rows at every chunk boundary and at
    a seed-row boundary are checked against the oracle.
    """
    m = 64
    b = synthetic.random_walk(1 << 20, 81).astype(np.float32)
    offs = np.array([0, 300_000, 300_100, 1 << 20])
    q = synthetic.random_walk(700_000 + m - 1, 82).astype(np.float32)
    dist, idx = join(mp, ctx, q, b, offs, m)
    edges = np.array([0, 1, 639, 640, 327_679, 327_680, 327_681, 655_359, 655_360, 655_361, 699_999])
    rows = np.unique(np.concatenate([edges, np.random.default_rng(4).choice(700_000, 40, replace=False)]))
    parity.check(dist, idx, q, b, offs, m, rows=rows, atol=1e-4)
    assert np.all((dist >= 0) & (dist <= 2 * math.sqrt(m) + 1e-9))


def _near_copies_case():
    """One dictionary segment holding seven copies of an ECG-like stretch plus one fixed white-noise pattern,
    the pattern's amplitude falling from copy to copy (0.2 of the stretch's std, 1.5e-5 less per copy, so the
    best copy comes last); the query embeds the unperturbed stretch. For most query windows inside it, the
    copies' windows at the same offset lie within 3.5e-5 of each other in correlation (distances about 0.9
    to 2, each copy 1e-4 to 3e-4 closer than the one before): all inside the plain kernel's near-tie width,
    and a few times the FP32 recurrence's own error apart."""
    m = 64
    rng = np.random.default_rng(2024)
    stretch = synthetic.ecg_like(200, 61).astype(np.float64)
    sd = float(np.std(stretch))
    pattern = rng.standard_normal(len(stretch))
    amps = 0.2 + 1.5e-5 * np.arange(7)[::-1]
    b = np.concatenate([stretch + a * sd * pattern for a in amps]).astype(np.float32)
    offs = np.array([0, len(b)], dtype=np.int64)
    q = synthetic.ecg_like(3000, 62).astype(np.float64)
    q[1000:1200] = stretch
    return q.astype(np.float32), b, offs, m


def _ilog2(x):
    return int(x).bit_length() - 1


@pytest.mark.parametrize("groups", [1, 3, 7, 40])
def test_results_do_not_depend_on_the_column_grouping(mp, tmp_path, groups):
    """Column groups are cut at chunk starts (every 16 windows from a segment's first window), so a window is
    scored in the same chunk with the same shift under any grouping: a tuning-cache line that forces the
    plain form to `groups` column groups gives the default join's results bit for bit."""
    b = synthetic.ecg_like(9000, 71).astype(np.float32)
    offs = np.array([0, 1234, 4321, 4999, 9000], dtype=np.int64)  # ragged segments
    q = synthetic.ecg_like(6000, 72).astype(np.float32)
    m = 96
    n_w = sum(int(offs[i + 1] - offs[i]) - m + 1 for i in range(len(offs) - 1))
    nq = len(q) - m + 1
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        ref_d, ref_i = join(mp, ctx, q, b, offs, m)
    finally:
        mp.mp_shutdown(ctx)
    cache = tmp_path / "groups.jsonl"
    cache.write_text('{"dtype": %d, "m": %d, "wlog": %d, "qlog": %d, "kernel": %d, "groups": %d, "ms": 0}\n'
                     % (mp.MP_F32, m, _ilog2(n_w), _ilog2(nq), mp.MP_KERNEL_PLAIN, groups))
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_AUTO, tune_cache=str(cache))
    try:
        d = mp.mp_dict_load(ctx, b, offs, [m])
        assert mp.mp_plan_join(ctx, d, mp.MP_F32, len(q), m)["column_groups"] == groups
        dist, idx = mp.mp_ab_join(ctx, d, q, m)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
    assert np.array_equal(dist, ref_d) and np.array_equal(idx, ref_i)
    parity.check(dist, idx, q, b, offs, m, rows=np.arange(0, nq, 41), atol=1e-4)


def test_near_tie_records_overflow_rescans_the_group(mp, tmp_path):
    """Seven near-tied chunks per query window in one column group: more than the plain kernel's record slots.
    The records overflow, the finalisation re-scores the whole column group for those windows, and every
    row still matches the oracle (1e-4, the plain path's tolerance). The context's counters show that the
    overflow path ran. A tuning-cache line pins the plain form to one column group for this shape (the
    default cost model spreads a join this small over many narrow groups, each holding one copy)."""
    q, b, offs, m = _near_copies_case()
    n_w, nq = len(b) - m + 1, len(q) - m + 1
    cache = tmp_path / "one_group.jsonl"
    cache.write_text('{"dtype": %d, "m": %d, "wlog": %d, "qlog": %d, "kernel": %d, "groups": 1, "ms": 0}\n'
                     % (mp.MP_F32, m, _ilog2(n_w), _ilog2(nq), mp.MP_KERNEL_PLAIN))
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_AUTO, tune_cache=str(cache))
    try:
        mp.mp_counters(ctx, reset=True)
        d = mp.mp_dict_load(ctx, b, offs, [m])
        assert mp.mp_plan_join(ctx, d, mp.MP_F32, len(q), m)["column_groups"] == 1
        dist, idx = mp.mp_ab_join(ctx, d, q, m)
        c = mp.mp_counters(ctx)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
    od, oi, od2 = oracle.ab_join(q, b, offs, m)
    rows = np.arange(1000, 1200 - m + 1)
    assert np.all(oi[rows] >= 6 * 200), "the best window lies in the last copy"
    # a wrong pick among the copies would miss the oracle's distance by the gap
    assert np.sum(od2[rows] - od[rows] > 1.2e-4) >= 40, "the copies' distances must differ by more than 1e-4"
    parity.check(dist, idx, q, b, offs, m, atol=1e-4, oracle_out=(od, oi, od2))
    assert c[mp.MP_COUNTER_OVERFLOW_ROWS] >= 50, c
    assert c[mp.MP_COUNTER_OVERFLOW_CHUNKS] > 0, c


@pytest.mark.parametrize("kernel", ["MP_KERNEL_TC_BF16X3", "MP_KERNEL_TC_TF32"])
def test_near_copies_tensor_core_forms(mp, kernel):
    """The same seven near-tied copies through the tensor-core forms: their records (63 slots) hold every
    copy, and each row matches the oracle within the tensor-core tolerance."""
    q, b, offs, m = _near_copies_case()
    ctx = mp.mp_init(device=0, kernel=getattr(mp, kernel))
    try:
        dist, idx = join(mp, ctx, q, b, offs, m)
    finally:
        mp.mp_shutdown(ctx)
    parity.check(dist, idx, q, b, offs, m, atol=1e-3)
