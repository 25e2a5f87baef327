"""The near-tie width of the plain kernel against the drift of its FP32 recurrence.

The plain join (Sec. 3.2's per-segment AB-join, run as a diagonal recurrence)
restarts every diagonal from a seed at most 32 lanes x 20 rows = 640 steps
earlier. Chunks whose approximate score lies within the near-tie width of the
running best are re-scored exactly, so that width must exceed the recurrence's
drift in correlation with a margin. This test models the kernel's arithmetic
(each step two fused multiply-adds in float32, the terms rounded to float32)
from exact seeds on the ECG-like benchmark data and measures the largest drift
against the same recurrence in float64.
"""
from __future__ import annotations

import os
import re

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAX_STEPS = 640


def _near_tie_width() -> float:
    with open(os.path.join(ROOT, "paper_2112_12965_gb300", "csrc", "mp_internal.cuh")) as f:
        return float(re.search(r"kNearRhoFP32\s*=\s*([0-9.eE+-]+)f", f.read()).group(1))


def _stats(x, m):
    x64 = x.astype(np.float64)
    win = sliding_window_view(x64, m)
    mu = win.mean(axis=1)
    return mu, 1.0 / np.sqrt(((win - mu[:, None]) ** 2).mean(axis=1))


def _terms(x, mu, m):
    # df[i] = (x[i+m-1] - x[i-1]) / 2, dg[i] = (x[i+m-1] - mu[i]) + (x[i-1] - mu[i-1])
    x64 = x.astype(np.float64)
    n = len(mu)
    df, dg = np.zeros(n), np.zeros(n)
    df[1:] = (x64[m:m + n - 1] - x64[:n - 1]) / 2
    dg[1:] = (x64[m:m + n - 1] - mu[1:]) + (x64[:n - 1] - mu[:-1])
    return df, dg


def _f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def _fma32(x, y, z):
    # float32 inputs: x * y is exact in float64, and the sum is rounded to float32 once
    return _f32(x * y + z)


def test_near_tie_width_covers_the_fp32_recurrence_drift():
    w = synthetic.workload("ecg_1m_m256", scale=1 / 16)
    m = w.m
    a = w.query.astype(np.float32)
    mua, isa = _stats(a, m)
    dfa, dga = _terms(a, mua, m)
    dfa32, dga32 = _f32(dfa), _f32(dga)
    worst = 0.0
    for s_i in range(0, len(w.offsets) - 1, 8):
        seg = w.dict_samples[w.offsets[s_i]:w.offsets[s_i + 1]].astype(np.float32)
        mub, isb = _stats(seg, m)
        dfb, dgb = _terms(seg, mub, m)
        dfb32, dgb32 = _f32(dfb), _f32(dgb)
        centred = sliding_window_view(seg.astype(np.float64), m) - mub[:, None]
        for r0 in range(0, len(mua) - MAX_STEPS, MAX_STEPS * 7):
            # exact seeds at row r0 for every column, then the diagonals run down
            c64 = centred @ (a[r0:r0 + m].astype(np.float64) - mua[r0])
            c32 = _f32(c64)
            for s in range(1, MAX_STEPS):
                r, k = r0 + s, len(c64)
                if k <= 1:
                    break
                # column c at depth s continues column c - 1 at depth s - 1
                g = slice(s, s + k - 1)
                c64 = c64[:-1] + dfa[r] * dgb[g] + dfb[g] * dga[r]
                c32 = _fma32(dfa32[r], dgb32[g], _fma32(dfb32[g], dga32[r], c32[:-1]))
                drift = np.abs(c32 - c64) * isa[r] * isb[g] / m
                worst = max(worst, float(drift.max()))
    width = _near_tie_width()
    assert 0.0 < worst < width / 8, (worst, width)
