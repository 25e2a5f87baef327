"""Benchmark of the dictionary AB-join on GB300.

Headline workload: ECG-like query of 2^20 samples (seed 2, 20 malformed beats)
against a dictionary of 64 segments x 1024 samples (seed 3), m = 256, float32
samples with FP64 window statistics. A step is one whole join (window
statistics, join kernel, finalisation with the exact distance of each pick).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--kernel plain|bf16x3|tf32|bf16|auto] [--serving-requests R]

Prints one JSON line (rank 0). With N > 1 (launched by torchrun) the query has
N times the headline's windows and is partitioned by query rows: every rank
joins its run of windows plus their m - 1 halo samples (weak scaling, no
data-path collective); the value is the total pairs of all ranks divided by
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ecg_1m_m256"
WORKLOAD_DESC = ("query 2^20 ECG-like samples (seed 2, 20 malformed beats) vs dictionary 64 segments x 1024 "
                 "samples (seed 3), m=256, float32 samples, FP64 window statistics")
METRIC = "AB-join pairs/s at m=256 (tensor-core vs plain kernel); p50/p99 serving latency"
L2_BYTES = 129 * 2**20
# The plain kernel's algorithmic work per (query window, dictionary window)
# pair: 2 FMAs of the covariance recurrence, 1 FMA for the score, 1
# compare-and-keep of the running maximum = 4 FP32-pipe lane instructions.
PLAIN_OPS_PER_PAIR = 4
# DRAM bytes of one k_plain launch on the full-size ECG workload (2^20 query
# samples, 64 x 1024 dictionary, m = 256), from one single-pass ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum: 672.09 MB read (the top seeds
# and the left seeds of the tensor cores) and 160.11 MB written (partial
# results and near-tie record headers). Valid for this kernel build (seeds from
# K2s and K2l, four-slot records, packed-multiply score fused with the
# recurrence step) and workload only.
PLAIN_DRAM_BYTES_FULL = 672.09e6 + 160.11e6
LANES_PER_SM = 128  # FP32 lanes per SM
# query windows per top seed of the FP32 plain kernel: one per warp, 32 lanes x 20 rows
SEED_STRIDE = 32 * 20


def shard_rows(n: int, m: int, world: int, rank: int):
    """Sample range [lo, hi) of rank's shard of a query of n samples.

    Query windows 0 .. n-m are split into `world` contiguous runs; a shard
    carries its windows' samples plus the m - 1 samples of halo they reach
    into, so the per-rank profiles concatenate to the whole profile with no
    exchange between ranks.
    """
    nq = max(0, n - m + 1)
    w_lo = nq * rank // world
    w_hi = nq * (rank + 1) // world
    if w_hi <= w_lo:
        return w_lo, w_lo
    return w_lo, w_hi + m - 1


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (all ranks get it); the identity for one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, target_s: float = 15.0):
    """Time the oracle (as it is) on a bounded sample of query windows."""
    import oracle

    oracle.build()
    nq = w.n_rows
    # calibrate on 256 rows (about 0.3 s, enough to amortise the oracle's start-up),
    # then size the sample for ~target_s seconds
    rows = np.arange(0, nq, max(1, nq // 256))[:256]
    t0 = time.perf_counter()
    oracle.ab_join(w.query, w.dict_samples, w.offsets, w.m, rows=rows)
    dt = time.perf_counter() - t0
    n_rows = int(max(256, min(nq, len(rows) * target_s / max(dt, 1e-6))))
    rows = np.linspace(0, nq - 1, n_rows).astype(np.int64)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.ab_join(w.query, w.dict_samples, w.offsets, w.m, rows=rows, nthreads=cores)
    dt = time.perf_counter() - t0
    pairs = n_rows * w.n_dict_windows
    # the same oracle on one thread, on a sample sized for about 3 s
    n1 = int(max(16, min(nq, n_rows * 3.0 / max(dt, 1e-6) / cores)))
    rows1 = np.linspace(0, nq - 1, n1).astype(np.int64)
    t0 = time.perf_counter()
    oracle.ab_join(w.query, w.dict_samples, w.offsets, w.m, rows=rows1, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_rows} evenly spaced of {nq} query windows, all {w.n_dict_windows} dictionary windows, "
                      f"{dt:.1f} s",
            "single_thread_value": n1 * w.n_dict_windows / dt1,
            "single_thread_sample": f"{n1} evenly spaced query windows, {dt1:.1f} s on 1 thread"}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, timed on this host's cores."""
    import synthetic

    if rank != 0:
        return
    w = synthetic.workload(WORKLOAD)
    import oracle

    oracle.build()
    nq = w.n_rows
    rows_per_step = 256
    # every core of the host, whatever OMP_NUM_THREADS says (torchrun sets it to 1)
    cores = os.cpu_count() or 1
    times = []
    for s in range(args.warmup + args.steps):
        rows = (np.arange(rows_per_step) * (nq // rows_per_step) + s) % nq
        t0 = time.perf_counter()
        oracle.ab_join(w.query, w.dict_samples, w.offsets, w.m, rows=rows, nthreads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    pairs = rows_per_step * w.n_dict_windows
    ms = 1e3 * float(np.mean(times))
    value = pairs / (ms / 1e3)
    # n_gpus is the launch's N, as in the other arm's line (this arm computes on the host's cores only)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "sample_rows_per_step": rows_per_step},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{rows_per_step} query windows per step, all {w.n_dict_windows} "
                                       "dictionary windows"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def roofline(kname, pairs, m, join_ms, peaks, peak_src, full_size=False, sms=152):
    """Roofline of the join kernel: ALU-issue bound (plain) or tensor bound (tcgen05).

    `traffic` (DRAM bytes per launch, from ncu) is known for the plain kernel on
    the full-size workload only; null otherwise."""
    if kname == "plain":
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak_ops = sms * LANES_PER_SM * mhz * 1e6 / 1e12  # T lane-instructions/s
        achieved = pairs * PLAIN_OPS_PER_PAIR / (join_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s",
                "frac": achieved / peak_ops, "traffic": PLAIN_DRAM_BYTES_FULL if full_size and PLAIN_DRAM_BYTES_FULL else None,
                "kernel": "k_plain",
                "peak_source": f"{sms} SMs x {LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz ({peak_src} max clock)",
                "ops_per_pair": PLAIN_OPS_PER_PAIR}
    tflops_peak = peaks.get("bf16_tflops", 1900.0)
    mult = 3 if kname == "bf16x3" else 1
    src = f"{peak_src} bf16 burst"
    if kname == "tf32":
        tflops_peak /= 2.0
        src += " / 2 (nominal TF32:BF16 ratio)"
    achieved = pairs * 2 * m * mult / (join_ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": tflops_peak, "unit": "TFLOP/s",
            "frac": achieved / tflops_peak, "traffic": None,
            "kernel": "k_tc<%d>" % {"bf16x3": 0, "tf32": 1, "bf16": 3}[kname],
            "peak_source": src, "flops_per_pair": 2 * m * mult}


def seed_roofline(w, seeds_ms, peaks, peak_src):
    """Tensor roofline of the plain join's top-seed kernel (K2s): one seed row per SEED_STRIDE
    query windows against every dictionary window, K = m, three TF32 products per term."""
    if seeds_ms <= 0:
        return None
    n_srows = -(-w.n_rows // SEED_STRIDE)
    flops = n_srows * w.n_dict_windows * 2 * w.m * 3
    peak = peaks.get("bf16_tflops", 1900.0) / 2.0
    achieved = flops / (seeds_ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "k_seed", "ms": seeds_ms, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "flops_per_launch": flops,
            "peak_source": f"{peak_src} bf16 burst / 2 (nominal TF32:BF16 ratio)"}


def left_seed_roofline(w, spans, left_ms, peaks, peak_src):
    """Tensor roofline of the plain join's left-seed kernel (K2l): every query window against
    the first window of every dictionary span (spans from mp_plan_join), K = m, three TF32
    products per term."""
    if left_ms <= 0 or spans <= 0:
        return None
    flops = w.n_rows * spans * 2 * w.m * 3
    peak = peaks.get("bf16_tflops", 1900.0) / 2.0
    achieved = flops / (left_ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "k_left_seed", "ms": left_ms, "spans": spans, "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "flops_per_launch": flops,
            "peak_source": f"{peak_src} bf16 burst / 2 (nominal TF32:BF16 ratio)"}


def kernel_id(mp, name):
    return {"plain": mp.MP_KERNEL_PLAIN, "bf16x3": mp.MP_KERNEL_TC_BF16X3, "tf32": mp.MP_KERNEL_TC_TF32,
            "bf16": mp.MP_KERNEL_TC_BF16,
            "auto": mp.MP_KERNEL_AUTO}[name]


def time_device_join(mp, ctx, d, w, steps, warmup, flush):
    """Per-step CUDA-event time of the whole join and per-phase event time."""
    import torch

    qt = torch.from_numpy(w.query).cuda()
    nq = w.n_rows
    dd = torch.empty(nq, dtype=torch.float64, device="cuda")
    di = torch.empty(nq, dtype=torch.int64, device="cuda")
    # A dedicated (non-default) stream: the library launches on it, and the
    # timing events are recorded on it.
    stream = torch.cuda.Stream()
    assert stream.cuda_stream != 0
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            mp.mp_ab_join_device(ctx, d, qt.data_ptr(), mp.MP_F32, len(w.query), w.m, dd.data_ptr(), di.data_ptr(),
                                 stream.cuda_stream)
        stream.synchronize()
        mp.mp_profile(ctx, True)
        mp.mp_profile_read(ctx, reset=True)
        step_ms = []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps (outside the timed events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mp.mp_ab_join_device(ctx, d, qt.data_ptr(), mp.MP_F32, len(w.query), w.m, dd.data_ptr(),
                                 di.data_ptr(), stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    phase_ms, phase_n = mp.mp_profile_read(ctx, reset=True)
    mp.mp_profile(ctx, False)
    return step_ms, phase_ms, phase_n, (dd, di)


def time_e2e(mp, ctx, d, w, steps, warmup):
    """End to end through mp_ab_join: pinned host query in, host result out, every step."""
    import torch

    q_pin = torch.from_numpy(w.query).pin_memory()
    nq = w.n_rows
    od = torch.empty(nq, dtype=torch.float64).pin_memory()
    oi = torch.empty(nq, dtype=torch.int64).pin_memory()
    qa, da, ia = q_pin.numpy(), od.numpy(), oi.numpy()
    import ctypes

    def once():
        rc = mp.lib.mp_ab_join(ctx, d, qa.ctypes.data, mp.MP_F32, len(qa), w.m, da.ctypes.data, ia.ctypes.data)
        if rc != 0:
            raise mp.MPError(rc, mp.mp_last_error())

    for _ in range(warmup):
        once()
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        once()
        t.append(time.perf_counter() - t0)
    return t, len(qa) * 4, nq * 16


def _device_join_timed(mp, ctx, d, q, m, reps=3):
    """Join a host query on the device; returns (dist, idx, join ms per call: the join kernel plus, for
    the plain form, its tensor-core seed kernel)."""
    import torch

    qt = torch.from_numpy(q).cuda()
    nq = len(q) - m + 1
    dd = torch.empty(nq, dtype=torch.float64, device="cuda")
    di = torch.empty(nq, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    mp.mp_ab_join_device(ctx, d, qt.data_ptr(), mp.MP_F32, len(q), m, dd.data_ptr(), di.data_ptr(), s.cuda_stream)
    s.synchronize()
    mp.mp_profile(ctx, True)
    mp.mp_profile_read(ctx, reset=True)
    for _ in range(reps):
        mp.mp_ab_join_device(ctx, d, qt.data_ptr(), mp.MP_F32, len(q), m, dd.data_ptr(), di.data_ptr(),
                             s.cuda_stream)
    s.synchronize()
    ms, n = mp.mp_profile_read(ctx, reset=True)
    mp.mp_profile(ctx, False)
    # a large join runs in several row chunks
    per_call = (ms[mp.MP_PHASE_JOIN] + ms[mp.MP_PHASE_SEEDS] + ms[mp.MP_PHASE_LEFT_SEEDS]) / reps
    _device_join_timed.last_phases = {"stats": ms[0] / reps, "join": ms[1] / reps, "finalize": ms[2] / reps,
                                      "seeds": ms[3] / reps, "left_seeds": ms[4] / reps}
    return dd.cpu().numpy(), di.cpu().numpy(), float(per_call)


def study_precision(mp, rows=256):
    """Per-result distance error of each join form against the FP64 oracle (transportation workload)."""
    import oracle
    import synthetic

    w = synthetic.workload("transport_4m_m512")
    r = np.linspace(0, w.n_rows - 1, rows).astype(np.int64)
    od, oi, od2 = oracle.ab_join(w.query, w.dict_samples, w.offsets, w.m, rows=r)
    ctx = mp.mp_init(device=0)
    out = {"study": "precision", "workload": "transportation-like query 2^22 (seed 4), dictionary 256 x 2048 "
           "(seed 5), m=512", "rows_checked": rows, "pairs": w.pairs, "forms": {}}
    try:
        d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
        for kname in ("plain", "bf16x3", "tf32", "bf16"):
            mp.mp_set_kernel(ctx, kernel_id(mp, kname))
            mp.mp_counters(ctx, reset=True)
            dist, idx, jm = _device_join_timed(mp, ctx, d, w.query, w.m, reps=2)
            ph = _device_join_timed.last_phases
            c = mp.mp_counters(ctx, reset=True) / 3  # three joins: a warm-up and two timed
            err = np.abs(dist[r] - od)
            uniq = (od2 - od) > 1e-3
            out["forms"][kname] = {
                "join_ms": jm, "pairs_per_s": w.pairs / (jm / 1e3), "phases_ms": ph,
                "step_pairs_per_s": w.pairs / (sum(ph.values()) / 1e3),
                "near_rows_per_join": float(c[mp.MP_COUNTER_NEAR_ROWS]),
                "near_chunks_per_join": float(c[mp.MP_COUNTER_NEAR_CHUNKS]),
                "overflow_rows_per_join": float(c[mp.MP_COUNTER_OVERFLOW_ROWS]),
                "abs_err_max": float(err.max()), "abs_err_p99": float(np.percentile(err, 99)),
                "abs_err_median": float(np.median(err)), "abs_err_mean": float(err.mean()),
                "index_match": float(np.mean(idx[r] == oi)),
                "index_match_where_gap_gt_1e-3": float(np.mean(idx[r][uniq] == oi[uniq])) if uniq.any() else None}
        mp.mp_dict_free(ctx, d)
    finally:
        mp.mp_shutdown(ctx)
    return out


def study_dict_vs_orig(mp, k_discords=200, with_tf32=False):
    """Join a 2^24 ECG-like query against the 128-segment dictionary and against the whole training series."""
    import synthetic

    wd = synthetic.workload("ecg_16m_m1024_dict")
    wo = synthetic.workload("ecg_16m_m1024_orig")
    m = wd.m
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN)
    out = {"study": "dictionary vs original", "workload": "ECG-like query 2^24 (seed 7, 200 malformed beats); "
           "dictionary 128 x 2048 cut from a normal-beat 2^22 training series (seed 6) vs that whole series; m=1024",
           "pairs_dict": wd.pairs, "pairs_orig": wo.pairs}
    try:
        dd = mp.mp_dict_load(ctx, wd.dict_samples, wd.offsets, [m])
        do = mp.mp_dict_load(ctx, wo.dict_samples, wo.offsets, [m])
        Ph, _, ms_d = _device_join_timed(mp, ctx, dd, wd.query, m, reps=1)
        P, _, ms_o = _device_join_timed(mp, ctx, do, wo.query, m, reps=1)
        e_max, _ = mp.mp_emax(ctx, dd, wo.dict_samples, m)
        diff = Ph - P
        ih, _, cert = mp.mp_top_discords(Ph, k_discords, m // 2, e_max)
        io, _, _ = mp.mp_top_discords(P, k_discords, m // 2)
        overlap = float(np.mean([np.min(np.abs(io - i)) <= m // 2 for i in ih])) if len(ih) else 0.0
        out.update({
            "join_ms_dict": ms_d, "join_ms_orig": ms_o, "speedup": ms_o / ms_d,
            "pairs_per_s_dict": wd.pairs / (ms_d / 1e3), "pairs_per_s_orig": wo.pairs / (ms_o / 1e3),
            "e_max": e_max, "max_P_hat_minus_P": float(diff.max()), "min_P_hat_minus_P": float(diff.min()),
            "mean_P_hat_minus_P": float(diff.mean()),
            "lemma1_holds": bool(np.all(diff >= -2e-4)), "lemma2_holds": bool(np.all(diff <= e_max + 2e-4)),
            "top_discord_overlap": overlap, "k_discords": len(ih), "top1_certified": cert})
        if with_tf32:
            mp.mp_set_kernel(ctx, mp.MP_KERNEL_TC_TF32)
            Pt, _, ms_t = _device_join_timed(mp, ctx, dd, wd.query, m, reps=1)
            out["tf32_dict_join_ms"] = ms_t
            out["tf32_vs_plain_max_abs_diff"] = float(np.max(np.abs(Pt - Ph)))
        mp.mp_dict_free(ctx, dd)
        mp.mp_dict_free(ctx, do)
    finally:
        mp.mp_shutdown(ctx)
    return out


def study_learn(mp, n_b=1 << 20, m=256, budget_frac=0.01, seed=6):
    """Algorithm 1 on the GPU for an ECG-like training series; streaming join throughput against the result."""
    import oracle
    import synthetic

    x = synthetic.ecg_like(n_b, seed).astype(np.float32)
    # up to 256 requests (stream appends) admitted at once, 128 per batched launch
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=256, max_batch=128)
    out = {"study": "dictionary learning (Algorithm 1) and streaming",
           "workload": f"ECG-like training series of {n_b} samples (seed {seed}, normal beats), m={m}, context k=1.5, "
                       f"memory budget {budget_frac:.0%} of the series"}
    try:
        nq = n_b - m + 1
        t0 = time.perf_counter()
        P, _ = mp.mp_self_join(ctx, x, m, (m + 1) // 2)
        t_sj = time.perf_counter() - t0
        t0 = time.perf_counter()
        segs, chosen, bound = mp.mp_learn_dictionary(ctx, x, m, 1.5, mp.MP_LEARN_MEMORY, budget_frac * n_b)
        t_learn = time.perf_counter() - t0
        samples = np.concatenate([x[a : a + L] for a, L in segs])
        offs = np.concatenate(([0], np.cumsum([L for _, L in segs])))
        d = mp.mp_dict_load(ctx, samples, offs, [m])
        e_max, _ = mp.mp_emax(ctx, d, x, m)
        # streaming: a fresh series arriving in appends of 1024 samples
        q = synthetic.ecg_like(1 << 20, seed + 1, n_malformed=20).astype(np.float32)
        st = mp.mp_stream_open(ctx, d, mp.MP_F32, m)
        t0 = time.perf_counter()
        n_win = 0
        for a in range(0, len(q), 1024):
            sd, _, _ = mp.mp_stream_append(st, q[a : a + 1024])
            n_win += len(sd)
        t_stream = time.perf_counter() - t0
        mp.mp_stream_close(st)
        # the same appends without waiting (mp_stream_submit: each append a serving request), up to
        # 1024 outstanding (the library admits 256 at once, 128 per batched launch); equal to the
        # synchronous appends' results
        st = mp.mp_stream_open(ctx, d, mp.MP_F32, m)
        t0 = time.perf_counter()
        live, outs, n_win_async = collections.OrderedDict(), [], 0
        for a in range(0, len(q), 1024):
            piece = q[a : a + 1024]
            od, oi = np.empty(len(piece)), np.empty(len(piece), dtype=np.int64)
            while True:
                try:
                    t, k, _ = mp.mp_stream_submit(st, piece, od, oi)
                    break
                except mp.MPError as e:  # admission queue full: wait for some
                    if e.code != mp.MP_E_BUSY:
                        raise
                    time.sleep(0.0001)
            outs.append((od, oi, k))
            n_win_async += k
            if t:
                live[t] = True
            while len(live) >= 1024:  # oldest first: appends finish roughly in order
                tk = next(iter(live))
                stt, _ = mp.mp_poll(ctx, tk)
                if stt == mp.MP_PENDING:
                    time.sleep(0)  # yield to the library's scheduler thread
                    continue
                if stt != mp.MP_DONE:
                    raise RuntimeError("stream append failed")
                del live[tk]
        mp.mp_drain(ctx, 600.0)
        for tk in list(live):
            stt, _ = mp.mp_poll(ctx, tk)
            if stt != mp.MP_DONE:
                raise RuntimeError("stream append failed")
        t_async = time.perf_counter() - t0
        mp.mp_stream_close(st)
        n_w = mp.mp_dict_windows(d, m)
        mp.mp_dict_free(ctx, d)
        # the float64 oracle's Algorithm 1 on a 1/32 sample (the same loop, for context)
        xs = x[: n_b // 32]
        t0 = time.perf_counter()
        oracle.learn_dictionary(xs, m, 1.5, "memory", budget_frac * len(xs))
        t_or = time.perf_counter() - t0
        out.update({
            "self_join_s": t_sj, "self_join_pairs_per_s": nq * (nq - m) / t_sj,
            "learn_s": t_learn, "iterations": len(chosen), "segments": len(segs),
            "dictionary_samples": int(offs[-1]), "error_bound_max_S": bound, "e_max_of_learned_dictionary": e_max,
            "profile_self_join_min_max": [float(np.min(P)), float(np.max(P))],
            "stream_appends_of_1024": int((len(q) + 1023) // 1024), "stream_windows": n_win,
            "stream_windows_per_s": n_win / t_stream, "stream_pairs_per_s": n_win * n_w / t_stream,
            "stream_submit_windows_per_s": n_win_async / t_async,
            "stream_submit_pairs_per_s": n_win_async * n_w / t_async,
            "oracle_learn_s_on_1_32": t_or, "oracle_cores": os.cpu_count()})
    finally:
        mp.mp_shutdown(ctx)
    return out


def serving_run(mp, n_requests=10000, loads=(0.5, 0.9), seed=11, pool_size=256, window=64):
    """The serving workload: 10,000 join requests, query lengths log-uniform in [2^10, 2^20] samples
    (random walk and ECG-like 50:50), m uniform in {64, 128, 256}, against 16 resident dictionaries of
    2^14..2^18 samples. First the capacity (a window of requests kept outstanding), then Poisson arrivals
    at each fraction of it; p50/p99 latency and throughput per load. Every request must succeed."""
    import synthetic

    if n_requests <= 0:
        return None
    rng = np.random.default_rng(seed)
    dicts = synthetic.serving_dictionaries(n_dicts=16, seed=100)
    # a pool of queries, log-uniform in [2^10, 2^20] samples, random walk / ECG-like 50:50
    pool = []
    for k in range(pool_size):
        n = int(2 ** rng.uniform(10, 20))
        sd = int(rng.integers(0, 2**31 - 1))
        q = synthetic.random_walk(n, sd) if k % 2 == 0 else synthetic.ecg_like(n, sd)
        pool.append(q.astype(np.float32))
    reqs = [(int(rng.integers(0, pool_size)), int(rng.integers(0, 16)), int(rng.choice([64, 128, 256])))
            for _ in range(n_requests)]
    ctx = mp.mp_init(device=0, kernel=mp.MP_KERNEL_PLAIN, max_inflight=16, max_batch=32)
    out = {"requests": n_requests,
           "mix": "query 2^U samples, U ~ U(10, 20), random walk / ECG-like 50:50 from a pool of "
                  f"{pool_size} series; m uniform in {{64, 128, 256}}; 16 resident dictionaries of 2^14..2^18 "
                  "samples cut into segments of 512..4096", "loads": {}}
    try:
        handles = [mp.mp_dict_load(ctx, b, offs, [64, 128, 256]) for b, offs in dicts]
        W = {(di, m): mp.mp_dict_windows(handles[di], m) for di in range(16) for m in (64, 128, 256)}

        def submit(r):
            q = pool[r[0]]
            nq = len(q) - r[2] + 1
            od, oi = np.empty(nq), np.empty(nq, dtype=np.int64)
            t = mp.mp_submit(ctx, handles[r[1]], q, r[2], od, oi)
            return t, (od, oi), nq * W[(r[1], r[2])]

        # capacity: keep `window` requests outstanding
        t0 = time.perf_counter()
        live, pairs, done = {}, 0, 0
        it = iter(reqs)
        exhausted = False
        while live or not exhausted:
            while not exhausted and len(live) < window:
                try:
                    r = next(it)
                except StopIteration:
                    exhausted = True
                    break
                t, bufs, pr = submit(r)
                live[t] = bufs
                pairs += pr
            for t in list(live):
                st, _ = mp.mp_poll(ctx, t)
                if st != mp.MP_PENDING:
                    if st != mp.MP_DONE:
                        raise RuntimeError(f"serving: request {t} failed")
                    del live[t]
                    done += 1
            time.sleep(0.0001)
        cap_s = time.perf_counter() - t0
        capacity = n_requests / cap_s
        out["capacity_rps"] = capacity
        out["capacity_pairs_per_s"] = pairs / cap_s
        for frac in loads:
            rate = frac * capacity
            arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
            lat, live = [], {}
            t0 = time.perf_counter()
            k = 0
            while k < n_requests or live:
                now = time.perf_counter() - t0
                while k < n_requests and arrivals[k] <= now:
                    t, bufs, _ = submit(reqs[k])
                    live[t] = bufs
                    k += 1
                for t in list(live):
                    st, l = mp.mp_poll(ctx, t)
                    if st != mp.MP_PENDING:
                        if st != mp.MP_DONE:
                            raise RuntimeError(f"serving: request {t} failed")
                        lat.append(l)
                        del live[t]
                time.sleep(0.0001)
            wall = time.perf_counter() - t0
            lat = np.array(lat) * 1e3
            out["loads"][f"{frac:.1f}x"] = {"offered_rps": rate, "throughput_rps": n_requests / wall,
                                            "p50_ms": float(np.percentile(lat, 50)),
                                            "p99_ms": float(np.percentile(lat, 99)),
                                            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}
        for h in handles:
            mp.mp_dict_free(ctx, h)
    finally:
        mp.mp_shutdown(ctx)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="plain", choices=["plain", "bf16x3", "tf32", "bf16", "auto"])
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--study", choices=["precision", "dict-vs-orig", "serving", "learn"], default=None,
                    help="run a study instead of the headline benchmark (one JSON line)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the query (profiling captures of a small case); 1.0 = the full workload")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__ as g

    g.build()
    import paper_2112_12965_gb300 as mp
    import synthetic

    if args.study:
        if args.study == "precision":
            res = study_precision(mp)
        elif args.study == "serving":
            res = dict(study="serving", **serving_run(mp))
        elif args.study == "learn":
            res = study_learn(mp)
        else:
            res = study_dict_vs_orig(mp, with_tf32=True)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return

    w = synthetic.workload(WORKLOAD, scale=args.scale)
    if world > 1:
        # weak scaling over the query-row partition: one ECG-like query of world x the headline's windows,
        # rank r joining its contiguous run of windows (plus their m - 1 halo samples); the per-rank
        # profiles concatenate to the whole profile with no exchange between ranks
        nq1 = len(w.query) - w.m + 1
        full = synthetic.ecg_like(world * nq1 + w.m - 1, 2, n_malformed=20 * world).astype(np.float32)
        lo, hi = shard_rows(len(full), w.m, world, rank)
        w.query = full[lo:hi]
    ctx = mp.mp_init(device=local_rank, kernel=kernel_id(mp, args.kernel))
    d = mp.mp_dict_load(ctx, w.dict_samples, w.offsets, [w.m])
    plan = mp.mp_plan_join(ctx, d, mp.MP_F32, len(w.query), w.m)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        step_ms, phase_ms, phase_n, _ = time_device_join(mp, ctx, d, w, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(float(np.sum(step_ms)), world, device="cuda")
    ms_per_step = total_ms / args.steps
    pairs = w.pairs  # this rank's
    total_pairs = world * nq1 * w.n_dict_windows if world > 1 else pairs  # the windows of all shards
    value = total_pairs * args.steps / (total_ms / 1e3)

    e2e_t, h2d, d2h = time_e2e(mp, ctx, d, w, max(3, args.steps // 2), 1)
    e2e_value = pairs / float(np.mean(e2e_t))

    peaks, peak_src = load_peaks()
    join_ms = phase_ms[mp.MP_PHASE_JOIN] / max(1, phase_n[mp.MP_PHASE_JOIN])
    clock = clk.summary()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    # the form the join ran (the autotuner's pick under --kernel auto)
    ran = {mp.MP_KERNEL_PLAIN: "plain", mp.MP_KERNEL_TC_BF16X3: "bf16x3", mp.MP_KERNEL_TC_TF32: "tf32",
           mp.MP_KERNEL_TC_BF16: "bf16"}[plan["kernel"]]
    roof = roofline(ran, pairs, w.m, join_ms, peaks, peak_src, full_size=args.scale == 1.0, sms=sms)
    # the other join forms on the same workload (same timing method)
    kernels = {}
    for kname in ("plain", "bf16x3", "tf32", "bf16"):
        if kname == args.kernel:
            sm, pm, pn = step_ms, phase_ms, phase_n
        else:
            mp.mp_set_kernel(ctx, kernel_id(mp, kname))
            sm, pm, pn, _ = time_device_join(mp, ctx, d, w, max(3, args.steps // 2), args.warmup, flush)
            mp.mp_set_kernel(ctx, kernel_id(mp, args.kernel))
        jm = pm[mp.MP_PHASE_JOIN] / max(1, pn[mp.MP_PHASE_JOIN])
        r = roofline(kname, pairs, w.m, jm, peaks, peak_src, sms=sms)
        kernels[kname] = {"pairs_per_s": pairs / (float(np.mean(sm)) / 1e3), "ms_per_step": float(np.mean(sm)),
                          "join_kernel_ms": jm, "join_pairs_per_s": pairs / (jm / 1e3),
                          "roofline_frac": r["frac"], "roofline_unit": r["unit"], "achieved": r["achieved"]}

    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "n_query_windows": w.n_rows, "n_dict_windows": w.n_dict_windows,
                   "pairs_per_step_per_gpu": pairs, "kernel": args.kernel, "scale": args.scale,
                   "l2": "flushed between timed steps (512 MB write outside the timed events)",
                   "parallelism": (f"one query of {world} x the windows, sharded by query rows over {world} GPUs "
                                   "(weak scaling, no data-path collective)") if world > 1 else "1 GPU"},
        "phases_ms": {"stats": phase_ms[0] / max(1, phase_n[0]), "seeds": phase_ms[3] / max(1, phase_n[3]),
                      "left_seeds": phase_ms[4] / max(1, phase_n[4]), "join": join_ms,
                      "finalize": phase_ms[2] / max(1, phase_n[2])},
        "roofline": roof,
        "seed_roofline": seed_roofline(w, phase_ms[3] / max(1, phase_n[3]), peaks, peak_src),
        "left_seed_roofline": left_seed_roofline(w, plan["spans"], phase_ms[4] / max(1, phase_n[4]), peaks,
                                                 peak_src),
        "plan": plan,
        "kernels": kernels,
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(np.sum(phase_n)),
        "clocks": clock,
    }
    mp.mp_dict_free(ctx, d)
    mp.mp_shutdown(ctx)
    if rank == 0:
        serving = serving_run(mp, args.serving_requests)
        if serving:
            # headline percentiles at half the capacity; the synchronous join's rate for comparison
            half = serving["loads"].get("0.5x", {})
            serving = {"p50_ms": half.get("p50_ms"), "p99_ms": half.get("p99_ms"), **serving,
                       "capacity_vs_sync_join": serving["capacity_pairs_per_s"] / value}
            line["serving"] = serving
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
