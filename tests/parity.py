"""Comparison of the GPU join with the CPU oracle, with the tolerances of the build.

* Index rule: the GPU's nearest-neighbour index equals the oracle's wherever
  the oracle's best and second-best distances differ by more than `gap`
  (1e-3). Elsewhere the GPU's index must be a valid dictionary window whose
  oracle distance is within `gap` of the oracle's best.
* Distance rule: |d_gpu - d_oracle| <= `atol` for every row (1e-4 for the
  FP32-accumulated plain path, 1e-3 for the tensor-core path, 1e-8 for
  float64 data). Rows with no dictionary window must be +inf / -1 on both.
"""
from __future__ import annotations

import numpy as np

import oracle


def valid_window(g: int, offsets: np.ndarray, m: int) -> bool:
    s = int(np.searchsorted(offsets, g, side="right")) - 1
    return 0 <= s < len(offsets) - 1 and g + m <= offsets[s + 1]


def check(dist, idx, query, dict_samples, offsets, m, rows=None, atol=1e-4, gap=1e-3, oracle_out=None):
    """Compare GPU (dist, idx) -- full length, or already restricted to `rows` -- with the oracle."""
    dist = np.asarray(dist)
    idx = np.asarray(idx)
    if rows is not None and len(dist) != len(rows):
        dist = dist[rows]
        idx = idx[rows]
    od, oi, od2 = oracle_out if oracle_out is not None else oracle.ab_join(query, dict_samples, offsets, m, rows=rows)
    none = oi < 0
    assert np.array_equal(idx[none], oi[none]) and np.all(np.isinf(dist[none])), "rows without windows"
    ok = ~none
    err = np.abs(dist[ok] - od[ok])
    worst = int(np.argmax(err)) if err.size else 0
    assert err.size == 0 or err.max() <= atol, (
        f"distance error {err.max():.3g} > {atol:.1g} at row {np.nonzero(ok)[0][worst]}")
    uniq = ok & ((od2 - od) > gap)
    bad = np.nonzero(uniq & (idx != oi))[0]
    assert bad.size == 0, f"{bad.size} index mismatches where the neighbour is unique, e.g. row {bad[:5]}"
    # ambiguous rows: the GPU's pick must be a valid window and nearly optimal
    amb = np.nonzero(ok & ~uniq & (idx != oi))[0]
    rr = np.arange(len(dist)) if rows is None else np.asarray(rows)
    q = np.asarray(query, dtype=np.float64)
    b = np.asarray(dict_samples, dtype=np.float64)
    for k in amb:
        g = int(idx[k])
        assert valid_window(g, offsets, m), f"row {rr[k]}: index {g} is not a valid window"
        i = int(rr[k])
        dg = oracle.pair_distance(q[i : i + m], b[g : g + m])
        assert dg <= od[k] + gap, f"row {i}: pick {g} at {dg} vs best {od[k]}"
    return dict(max_err=float(err.max()) if err.size else 0.0,
                p99_err=float(np.percentile(err, 99)) if err.size else 0.0,
                n_rows=int(len(dist)), n_ambiguous=int((ok & ~uniq).sum()), n_amb_mismatch=int(amb.size))
