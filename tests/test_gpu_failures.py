"""Failure paths of the library, provoked on the host (needs a GB300 for the library itself).

No test faults, traps or hangs the GPU. Failures are made on the host: a
memory budget below one request, allocations that a testing hook makes fail,
a full admission queue, and a bound on the tensor-core kernel's waits that is
too short for its work (the kernel then gives up, records the error, waits for
its own tensor-core work and frees its tensor memory; the context stays
usable). After each failure the context must still join correctly.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import parity
import synthetic

pytestmark = pytest.mark.gpu


def _small_case(m=64):
    b = synthetic.ecg_like(6000, 41).astype(np.float32)
    offs = np.array([0, 3000, 6000], dtype=np.int64)
    q = synthetic.ecg_like(4000, 42).astype(np.float32)
    return q, b, offs, m


def _wait(mp, ctx, ticket, timeout_s=60.0):
    t_end = time.time() + timeout_s
    while time.time() < t_end:
        state, lat = mp.mp_poll(ctx, ticket)
        if state != mp.MP_PENDING:
            return state
        time.sleep(0.001)
    raise AssertionError("request did not finish")


def test_request_above_the_memory_budget_is_refused(mp):
    q, b, offs, m = _small_case()
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, mem_budget=1 << 16)
    try:
        d = mp.mp_dict_load(ctx, b, offs, [m])
        nq = len(q) - m + 1
        od, oi = np.zeros(nq), np.zeros(nq, dtype=np.int64)
        with pytest.raises(mp.MPError) as e:
            mp.mp_submit(ctx, d, q, m, od, oi)
        assert e.value.code == mp.MP_E_NOMEM and "budget" in str(e.value)
        # the context still joins
        dist, idx = mp.mp_ab_join(ctx, d, q, m)
        parity.check(dist, idx, q, b, offs, m, rows=np.arange(0, nq, 37), atol=1e-4)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_injected_allocation_failures_fail_only_their_requests(mp):
    q, b, offs, m = _small_case()
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=1)
    try:
        d = mp.mp_dict_load(ctx, b, offs, [m])
        nq = len(q) - m + 1
        mp.mp_test_hook(ctx, mp.MP_HOOK_FAIL_ALLOC, 2)
        outs = [(np.full(nq, -1.0), np.full(nq, -7, dtype=np.int64)) for _ in range(3)]
        tickets = [mp.mp_submit(ctx, d, q, m, od, oi) for od, oi in outs]
        states = [_wait(mp, ctx, t) for t in tickets]
        assert states == [mp.MP_FAILED, mp.MP_FAILED, mp.MP_DONE], states
        ref_d, ref_i = mp.mp_ab_join(ctx, d, q, m)
        assert np.array_equal(outs[2][0], ref_d) and np.array_equal(outs[2][1], ref_i)
        # failed requests released their dictionary reference: it can be freed
        mp.mp_drain(ctx, 30.0)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_full_admission_queue_refuses_then_recovers(mp):
    b = synthetic.ecg_like(1 << 16, 43).astype(np.float32)
    offs = np.array([0, 1 << 15, 1 << 16], dtype=np.int64)
    m = 256
    big = synthetic.ecg_like(1 << 20, 44).astype(np.float32)  # keeps the one slot busy for a while
    small = synthetic.ecg_like(3000, 45).astype(np.float32)
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=1, max_pending=2)
    try:
        d = mp.mp_dict_load(ctx, b, offs, [m])
        bufs, tickets, refused = [], [], 0
        for k in range(12):
            qk = big if k == 0 else small
            nq = len(qk) - m + 1
            od, oi = np.zeros(nq), np.zeros(nq, dtype=np.int64)
            try:
                tickets.append(mp.mp_submit(ctx, d, qk, m, od, oi))
                bufs.append((od, oi, qk))
            except mp.MPError as e:
                assert e.code == mp.MP_E_BUSY and "max_pending" in str(e)
                refused += 1
        assert refused > 0, "the queue never filled"
        assert all(_wait(mp, ctx, t) == mp.MP_DONE for t in tickets)
        # after the queue drains, submissions are admitted again, with correct results
        nq = len(small) - m + 1
        od, oi = np.zeros(nq), np.zeros(nq, dtype=np.int64)
        t = mp.mp_submit(ctx, d, small, m, od, oi)
        assert _wait(mp, ctx, t) == mp.MP_DONE
        ref_d, ref_i = mp.mp_ab_join(ctx, d, small, m)
        assert np.array_equal(od, ref_d) and np.array_equal(oi, ref_i)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


@pytest.mark.parametrize("kernel", ["MP_KERNEL_TC_BF16X3", "MP_KERNEL_TC_TF32"])
def test_tensor_core_wait_timeout_is_reported(mp, kernel):
    """A wait bound of one clock: the tensor-core join's roles give up on each other at once."""
    import torch

    q, b, offs, m = _small_case()
    ctx = mp.mp_init(device=0, kernel=getattr(mp, kernel))
    try:
        d = mp.mp_dict_load(ctx, b, offs, [m])
        ref_d, ref_i = mp.mp_ab_join(ctx, d, q, m)
        mp.mp_test_hook(ctx, mp.MP_HOOK_TC_WAIT, 1)
        with pytest.raises(mp.MPError) as e:
            mp.mp_ab_join(ctx, d, q, m)
        assert e.value.code == mp.MP_E_TIMEOUT
        qt = torch.from_numpy(q).cuda()
        nq = len(q) - m + 1
        dd = torch.zeros(nq, dtype=torch.float64, device="cuda")
        di = torch.zeros(nq, dtype=torch.int64, device="cuda")
        s = torch.cuda.Stream()
        mp.mp_ab_join_device(ctx, d, qt.data_ptr(), mp.MP_F32, len(q), m, dd.data_ptr(), di.data_ptr(), s.cuda_stream)
        s.synchronize()
        assert torch.all(torch.isnan(dd)).item() and torch.all(di == -1).item()
        # back to the default bound: the same context joins correctly again
        mp.mp_test_hook(ctx, mp.MP_HOOK_TC_WAIT, 0)
        dist, idx = mp.mp_ab_join(ctx, d, q, m)
        assert np.array_equal(dist, ref_d) and np.array_equal(idx, ref_i)
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
