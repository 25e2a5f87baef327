"""mp_ab_join_noalloc: the join for callers that must not allocate device memory.

Services that reserve all GPU memory up front, or applications whose own
allocator owns the device, cannot let a library call cudaMalloc while a
request is served. mp_ab_join_noalloc uses one fixed scratch array inside the
library instead of the context's workspace. These checks call it through the
C ABI and compare it with the regular device join (mp_ab_join_device), within
the plain path's parity tolerance, on two calls in a row with different
queries (the second call finds the first call's data in the shared array).
This file is collected last so that a failure here comes after every other
test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

import parity
import synthetic

pytestmark = pytest.mark.gpu


def _device_join(mp, torch, ctx, d, fn, q, m, stream):
    qt = torch.from_numpy(q).cuda()
    nq = len(q) - m + 1
    dist = torch.full((nq,), float("nan"), dtype=torch.float64, device="cuda")
    idx = torch.full((nq,), -7, dtype=torch.int64, device="cuda")
    fn(ctx, d, qt.data_ptr(), mp.MP_F32, len(q), m, dist.data_ptr(), idx.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return dist.cpu().numpy(), idx.cpu().numpy()


def test_noalloc_join_matches_device_join_on_two_calls(mp):
    import torch

    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        w = synthetic.workload("ecg_1m_m256", scale=1 / 4)  # 262,017 query windows, below the 2^19 limit
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        stream = torch.cuda.Stream()
        queries = [w.query, synthetic.ecg_like(len(w.query) - 4096, 77, n_malformed=5).astype(np.float32)]
        for q in queries:
            ref_d, ref_i = _device_join(mp, torch, ctx, d, mp.mp_ab_join_device, q, w.m, stream)
            got_d, got_i = _device_join(mp, torch, ctx, d, mp.mp_ab_join_noalloc, q, w.m, stream)
            assert np.all(np.isfinite(got_d)) and np.all(got_i >= 0)
            np.testing.assert_allclose(got_d, ref_d, rtol=0, atol=1e-4)
            diff = got_i != ref_i
            # a different pick is allowed only between near-tied windows
            assert diff.mean() < 1e-3
            assert np.all(np.abs(got_d[diff] - ref_d[diff]) <= 1e-4)
            rows = np.random.default_rng(len(q)).choice(len(got_d), 96, replace=False)
            parity.check(got_d, got_i, q, w.dict_samples, w.offsets, w.m, rows=rows, atol=1e-4)

        # beyond the stated maximum: a clear error, nothing launched
        big = np.zeros((1 << 19) + w.m, dtype=np.float32)
        with pytest.raises(mp.MPError) as e:
            _device_join(mp, torch, ctx, d, mp.mp_ab_join_noalloc, big, w.m, stream)
        assert e.value.code == mp.MP_E_ARG and "limit" in str(e.value)
        # statistics for another m would have to be allocated: refused
        with pytest.raises(mp.MPError) as e:
            _device_join(mp, torch, ctx, d, mp.mp_ab_join_noalloc, w.query[:5000], 128, stream)
        assert e.value.code == mp.MP_E_ARG
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)


def test_noalloc_join_allocates_no_device_memory(mp):
    """The defining property: after the first call on the device (which resolves the scratch array's address),
    a call leaves the device's free memory unchanged. A regular join on a fresh context, by contrast, grows
    the context's workspace."""
    import torch

    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    try:
        w = synthetic.workload("ecg_1m_m256", scale=1 / 16)
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        qt = torch.from_numpy(w.query).cuda()
        nq = len(w.query) - w.m + 1
        dist = torch.empty(nq, dtype=torch.float64, device="cuda")
        idx = torch.empty(nq, dtype=torch.int64, device="cuda")
        stream = torch.cuda.Stream()

        def call(fn):
            fn(ctx, d, qt.data_ptr(), mp.MP_F32, len(w.query), w.m, dist.data_ptr(), idx.data_ptr(),
               stream.cuda_stream)
            stream.synchronize()

        call(mp.mp_ab_join_noalloc)  # first call on the device
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            call(mp.mp_ab_join_noalloc)
        assert torch.cuda.mem_get_info()[0] == free0
        call(mp.mp_ab_join_device)  # the context's workspace: allocated now
        assert torch.cuda.mem_get_info()[0] < free0
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
