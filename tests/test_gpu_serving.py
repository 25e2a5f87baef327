"""Serving path (mp_submit / mp_poll): continuous batching on the GPU (needs a GB300)."""
from __future__ import annotations

import time

import numpy as np
import pytest

import parity
import synthetic

pytestmark = pytest.mark.gpu


def wait(mp, ctx, tickets, timeout=120.0):
    t_end = time.time() + timeout
    lat = {}
    left = set(tickets)
    while left:
        for t in list(left):
            st, l = mp.mp_poll(ctx, t)
            if st != mp.MP_PENDING:
                assert st == mp.MP_DONE, f"request {t} failed"
                lat[t] = l
                left.discard(t)
        assert time.time() < t_end, "serving timed out"
        time.sleep(0.0005)
    return lat


def make_mix(n_req=24, seed=0):
    dicts = synthetic.serving_dictionaries(n_dicts=4, seed=100, min_log2=12, max_log2=14)
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        n = int(2 ** rng.uniform(10, 14))
        m = int(rng.choice([64, 128, 256]))
        q = (synthetic.random_walk(n, 1000 + k) if k % 2 else synthetic.ecg_like(n, 1000 + k)).astype(np.float32)
        reqs.append((int(rng.integers(0, len(dicts))), q, m))
    return dicts, reqs


def test_serving_matches_sync_join_and_is_mix_invariant(mp):
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=6, max_batch=8)
    try:
        dicts, reqs = make_mix()
        handles = [mp.mp_dict_load(ctx, b, offs, [64, 128, 256]) for b, offs in dicts]
        # alone: one request at a time through the serving path
        alone = []
        for di, q, m in reqs:
            nq = len(q) - m + 1
            od, oi = np.empty(nq), np.empty(nq, dtype=np.int64)
            t = mp.mp_submit(ctx, handles[di], q, m, od, oi)
            wait(mp, ctx, [t])
            alone.append((od, oi))
        # in the mix: all submitted at once, batched and overlapped
        outs, tickets = [], []
        for di, q, m in reqs:
            nq = len(q) - m + 1
            od, oi = np.empty(nq), np.empty(nq, dtype=np.int64)
            outs.append((od, oi))
            tickets.append(mp.mp_submit(ctx, handles[di], q, m, od, oi))
        lat = wait(mp, ctx, tickets)
        assert len(lat) == len(reqs) and all(v >= 0 for v in lat.values())
        for (od, oi), (ad, ai), (di, q, m) in zip(outs, alone, reqs):
            assert np.array_equal(oi, ai) and np.array_equal(od, ad), "result changed in the mix"
            sd, si = mp.mp_ab_join(ctx, handles[di], q, m)
            np.testing.assert_allclose(od, sd, atol=1e-4, rtol=0)
            b, offs = dicts[di]
            rows = np.arange(0, len(od), max(1, len(od) // 64))
            parity.check(od, oi, q, b, offs, m, rows=rows, atol=1e-4)
        # a dictionary referenced by queued work cannot be freed
        di, q, m = reqs[0]
        big = np.tile(q, 64)
        od, oi = np.empty(len(big) - m + 1), np.empty(len(big) - m + 1, dtype=np.int64)
        t = mp.mp_submit(ctx, handles[di], big, m, od, oi)
        with pytest.raises(mp.MPError) as e:
            mp.mp_dict_free(ctx, handles[di])
        assert e.value.code in (mp.MP_E_BUSY,)
        wait(mp, ctx, [t])
        mp.mp_drain(ctx, 30.0)
        for h in handles:
            mp.mp_dict_free(ctx, h)
    finally:
        mp.mp_shutdown(ctx)


def test_serving_large_requests_match_sync_join(mp):
    """Requests of the serving benchmark's largest sizes (queries and dictionaries of up to 2^18 samples),
    submitted together: each result matches the synchronous join and, on sampled rows, the oracle. The
    batched kernel's geometry (its own rows per lane and column groups) must fit the memory the request was
    given at submission."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=8, max_batch=16)
    try:
        dicts = synthetic.serving_dictionaries(n_dicts=3, seed=140, min_log2=16, max_log2=18)
        handles = [mp.mp_dict_load(ctx, b, offs, [64, 128, 256]) for b, offs in dicts]
        rng = np.random.default_rng(5)
        reqs, outs, tickets = [], [], []
        for k in range(8):
            n = int(2 ** rng.uniform(15, 18))
            m = int(rng.choice([64, 128, 256]))
            q = (synthetic.random_walk(n, 3000 + k) if k % 2 else synthetic.ecg_like(n, 3000 + k)).astype(np.float32)
            di = int(rng.integers(0, len(dicts)))
            od, oi = np.empty(n - m + 1), np.empty(n - m + 1, dtype=np.int64)
            reqs.append((di, q, m))
            outs.append((od, oi))
            tickets.append(mp.mp_submit(ctx, handles[di], q, m, od, oi))
        wait(mp, ctx, tickets, timeout=300.0)
        for (od, oi), (di, q, m) in zip(outs, reqs):
            sd, _ = mp.mp_ab_join(ctx, handles[di], q, m)
            np.testing.assert_allclose(od, sd, atol=1e-4, rtol=0)
            b, offs = dicts[di]
            rows = np.unique(np.concatenate([np.arange(0, len(od), max(1, len(od) // 12)), [len(od) - 1]]))
            parity.check(od, oi, q, b, offs, m, rows=rows, atol=1e-4)
        mp.mp_drain(ctx, 60.0)
        for h in handles:
            mp.mp_dict_free(ctx, h)
    finally:
        mp.mp_shutdown(ctx)


def test_drain_returns_only_after_every_result_is_written(mp):
    """mp_drain must not return while a batch is being launched (its outputs unwritten)."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=4, max_batch=4)
    try:
        b, offs = synthetic.serving_dictionaries(n_dicts=1, seed=300, min_log2=12, max_log2=12)[0]
        h = mp.mp_dict_load(ctx, b, offs, [64])
        for rnd in range(5):
            outs = []
            for k in range(40):
                q = synthetic.random_walk(2000 + 37 * k, 7000 + 100 * rnd + k).astype(np.float32)
                od = np.full(len(q) - 63, np.nan)
                oi = np.full(len(q) - 63, -7, dtype=np.int64)
                outs.append((od, oi, mp.mp_submit(ctx, h, q, 64, od, oi)))
            mp.mp_drain(ctx, 60.0)
            for od, oi, t in outs:
                assert np.all(np.isfinite(od)) and np.all(oi >= 0), "drain returned before a result was written"
                st, _ = mp.mp_poll(ctx, t)
                assert st == mp.MP_DONE
        mp.mp_dict_free(ctx, h)
    finally:
        mp.mp_shutdown(ctx)


def test_sync_joins_while_batches_launch(mp):
    """The scheduler enqueues a batch's copies and launches without the context lock, so synchronous joins
    (which hold it) run while batches are being launched and executed. Both must give the results each gives
    alone: the serving results equal the synchronous join of the same query, bit for bit."""
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=16, max_batch=8)
    try:
        dicts, reqs = make_mix(n_req=48, seed=3)
        handles = [mp.mp_dict_load(ctx, b, offs, [64, 128, 256]) for b, offs in dicts]
        ref = [mp.mp_ab_join(ctx, handles[di], q, m) for di, q, m in reqs]
        outs, tickets = [], []
        for k, (di, q, m) in enumerate(reqs):
            nq = len(q) - m + 1
            od, oi = np.empty(nq), np.empty(nq, dtype=np.int64)
            tickets.append(mp.mp_submit(ctx, handles[di], q, m, od, oi))
            outs.append((od, oi))
            if k % 4 == 0:  # a synchronous join between submissions, while earlier batches run
                j = (k * 7) % len(reqs)
                d2, i2 = mp.mp_ab_join(ctx, handles[reqs[j][0]], reqs[j][1], reqs[j][2])
                assert np.array_equal(d2, ref[j][0]) and np.array_equal(i2, ref[j][1])
        wait(mp, ctx, tickets)
        for (od, oi), (rd, ri) in zip(outs, ref):
            assert np.array_equal(od, rd) and np.array_equal(oi, ri)
        for h in handles:
            mp.mp_dict_free(ctx, h)
    finally:
        mp.mp_shutdown(ctx)
