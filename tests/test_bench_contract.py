"""Host-side parts of bench.py's JSON contract (no GPU): the CPU baseline, the
reference arm's line and the roofline objects."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

import bench
import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_baseline_reports_all_cores_and_one_thread():
    w = synthetic.workload("ecg_1m_m256", scale=1 / 64)
    cb = bench.cpu_baseline(w, target_s=0.3)
    assert cb["kind"] == "oracle" and cb["unit"] == "pairs/s"
    assert cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["single_thread_value"] > 0
    assert "query windows" in cb["sample"] and "1 thread" in cb["single_thread_sample"]


def test_roofline_objects():
    peaks = {"bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    pairs, m = 1_000_000_000, 256
    plain_full = bench.roofline("plain", pairs, m, 1.0, peaks, "test", full_size=True)
    plain_small = bench.roofline("plain", pairs, m, 1.0, peaks, "test", full_size=False)
    # 4 lane instructions per pair over 1 ms, against 152 SMs x 128 lanes x 2000 MHz
    assert plain_full["bound"] == "alu"
    assert plain_full["achieved"] == pytest.approx(4e9 / 1e-3 / 1e12)
    assert plain_full["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert plain_full["frac"] == pytest.approx(plain_full["achieved"] / plain_full["peak"])
    # the measured DRAM traffic belongs to the full-size workload only
    assert plain_full["traffic"] == bench.PLAIN_DRAM_BYTES_FULL and plain_small["traffic"] is None
    assert plain_full["peak"] == pytest.approx(152 * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12)
    tc = bench.roofline("bf16x3", pairs, m, 1.0, peaks, "test")
    assert tc["bound"] == "tensor" and tc["flops_per_pair"] == 2 * m * 3 and tc["traffic"] is None
    tf = bench.roofline("tf32", pairs, m, 1.0, peaks, "test")
    assert tf["peak"] == pytest.approx(1000.0) and tf["flops_per_pair"] == 2 * m
    b1 = bench.roofline("bf16", pairs, m, 1.0, peaks, "test")
    assert b1["peak"] == pytest.approx(2000.0) and b1["flops_per_pair"] == 2 * m and b1["kernel"] == "k_tc<3>"
    assert tc["kernel"] == "k_tc<0>" and tf["kernel"] == "k_tc<1>"


def test_seed_rooflines():
    peaks = {"bf16_tflops": 2000.0}
    w = synthetic.workload("ecg_1m_m256", scale=1 / 64)
    top = bench.seed_roofline(w, 1.0, peaks, "test")
    # one seed row per 640 query windows against every dictionary window, three TF32 products
    assert top["flops_per_launch"] == -(-w.n_rows // 640) * w.n_dict_windows * 2 * w.m * 3
    assert top["peak"] == pytest.approx(1000.0)
    left = bench.left_seed_roofline(w, 160, 0.5, peaks, "test")
    # every query window against the first window of each of 160 spans
    assert left["flops_per_launch"] == w.n_rows * 160 * 2 * w.m * 3
    assert left["achieved"] == pytest.approx(left["flops_per_launch"] / 0.5e-3 / 1e12)
    assert bench.left_seed_roofline(w, 0, 0.5, peaks, "test") is None
    assert bench.seed_roofline(w, 0.0, peaks, "test") is None


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "pairs/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
