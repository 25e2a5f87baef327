"""CPU float64 oracle for the dictionary AB-join -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package. The GPU library never calls it, and it
imports nothing from the GPU package.

The arithmetic lives in ``mp_oracle.c`` (plain C, float64, OpenMP over query
windows), which follows the paper's definitions and Algorithm 2; this module
only compiles it with gcc and marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmporacle.so")
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH, extra_flags=()) -> str:
    """Compile ``mp_oracle.c`` into a shared library (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", *extra_flags, src, "-o", out, "-lm"]
        subprocess.run(cmd, check=True)
    return out


def load(path: Optional[str] = None):
    """Load (building first if needed) and type the oracle library."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    p = path or build()
    lib = ctypes.CDLL(p)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.mpo_window_stats.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, dp, dp, u8p]
    lib.mpo_window_stats.restype = ctypes.c_int
    lib.mpo_pair_distance.argtypes = [dp, dp, ctypes.c_int32]
    lib.mpo_pair_distance.restype = ctypes.c_double
    lib.mpo_ab_join.argtypes = [dp, ctypes.c_int64, dp, i64p, ctypes.c_int32, ctypes.c_int32,
                                i64p, ctypes.c_int64, dp, i64p, dp, ctypes.c_int]
    lib.mpo_ab_join.restype = ctypes.c_int
    lib.mpo_self_join.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, dp, i64p, ctypes.c_int]
    lib.mpo_self_join.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _f64(x) -> np.ndarray:
    # float32 samples widen exactly to float64: the oracle sees the same values
    # the GPU path sees.
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _ptr(x: np.ndarray, t):
    return x.ctypes.data_as(ctypes.POINTER(t))


def window_stats(x, m: int, lib=None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Per-window mean, population std and constant flag (two-pass, float64)."""
    lib = lib or load()
    x = _f64(x)
    nw = len(x) - m + 1
    mu = np.empty(nw)
    sd = np.empty(nw)
    cst = np.empty(nw, dtype=np.uint8)
    rc = lib.mpo_window_stats(_ptr(x, ctypes.c_double), len(x), m, _ptr(mu, ctypes.c_double),
                              _ptr(sd, ctypes.c_double), _ptr(cst, ctypes.c_uint8))
    if rc != 0:
        raise ValueError(f"mpo_window_stats failed ({rc})")
    return mu, sd, cst.astype(bool)


def pair_distance(x, y, lib=None) -> float:
    """z-normalised Euclidean distance of two equal-length windows."""
    lib = lib or load()
    x = _f64(x)
    y = _f64(y)
    assert len(x) == len(y)
    return float(lib.mpo_pair_distance(_ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), len(x)))


def ab_join(query, dict_samples, offsets, m: int, rows=None, nthreads: int = 0, lib=None):
    """Dictionary AB-join (Algorithm 2) of ``query`` against the segments.

    Returns ``(dist, idx, dist2)`` for the requested rows (all rows if
    ``rows`` is None): nearest-neighbour distance, global window index of the
    neighbour, and the smallest distance over every other window.
    """
    lib = lib or load()
    a = _f64(query)
    b = _f64(dict_samples) if len(dict_samples) else np.zeros(1)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    nq = len(a) - m + 1
    if rows is None:
        rows_arr = None
        nr = nq
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nr = len(rows_arr)
    dist = np.empty(nr)
    idx = np.empty(nr, dtype=np.int64)
    dist2 = np.empty(nr)
    rc = lib.mpo_ab_join(_ptr(a, ctypes.c_double), len(a), _ptr(b, ctypes.c_double), _ptr(offs, ctypes.c_int64),
                         len(offs) - 1, m,
                         None if rows_arr is None else _ptr(rows_arr, ctypes.c_int64), nr,
                         _ptr(dist, ctypes.c_double), _ptr(idx, ctypes.c_int64), _ptr(dist2, ctypes.c_double),
                         int(nthreads))
    if rc != 0:
        raise ValueError(f"mpo_ab_join failed ({rc})")
    return dist, idx, dist2


def ab_join_corr(query, dict_samples, offsets, m: int, rows=None, nthreads: int = 0, lib=None):
    """The join reported as a bounded similarity (Sec. 2.1 names the Pearson
    correlation coefficient as the alternative to the distance).

    For each row the largest rho over the dictionary windows, with
    rho = 1 - d^2 / (2m): for z-normalised windows of unit population
    variance, ||z_a - z_b||^2 = 2m - 2 sum_k z_a z_b = 2m (1 - r), so rho is
    Pearson's r when neither window is constant. Under the zero-vector
    convention for constant windows it is 0.5 between a constant and a
    non-constant window and 1 between two constant ones. The largest rho is
    the smallest d, so the index is the join's. Returns ``(rho, idx)``;
    rows without a dictionary window get -inf / -1.
    """
    d, i, _ = ab_join(query, dict_samples, offsets, m, rows=rows, nthreads=nthreads, lib=lib)
    rho = np.where(i >= 0, 1.0 - d * d / (2.0 * m), -np.inf)
    return rho, i


def self_join(series, m: int, excl: int, nthreads: int = 0, lib=None):
    """Self-join matrix profile (Algorithm 1's P_B): nearest window outside +-excl. Returns (dist, idx)."""
    lib = lib or load()
    a = _f64(series)
    nq = len(a) - m + 1
    dist = np.empty(nq)
    idx = np.empty(nq, dtype=np.int64)
    rc = lib.mpo_self_join(_ptr(a, ctypes.c_double), len(a), m, int(excl), _ptr(dist, ctypes.c_double),
                           _ptr(idx, ctypes.c_int64), int(nthreads))
    if rc != 0:
        raise ValueError(f"mpo_self_join failed ({rc})")
    return dist, idx


def learn_dictionary(t_b, m: int, k_context: float = 1.5, term: str = "memory", term_value: float = 0.0,
                     max_elements: int = 1 << 30, lib=None):
    """Dictionary learning, Algorithm 1 (Sec. 3.1), step by step in float64.

    P_B is the self-join with trivial matches |g - i| < ceil(m/2) left out
    (line 3). Each iteration takes j = argmin (P_B - S) outside the zones
    [j' - m/2, j' + m/2) of the windows taken before (lines 7-11, S = 0 at
    first, lowest index on ties), adds T_B[j : j + m] with
    floor((k - 1) m / 2) samples of context on each side (line 12), folds the
    distance profile of T_B against T_B[j : j + m] into S by an element-wise
    minimum (lines 15-19), and stops at the terminal condition (lines 13-14):
    ``term="memory"`` once the merged elements hold >= term_value samples,
    ``term="emax"`` once max(S) <= term_value; or after max_elements, or when
    no window is left. Overlapping elements are merged (Fig. 5).

    Returns ``(segments, chosen, err_bound)``: the merged elements as
    (start, length) pairs, the taken windows in order, and max(S) at the end.
    """
    lib = lib or load()
    x = _f64(t_b)
    n = len(x)
    nq = n - m + 1
    P, _ = self_join(x, m, (m + 1) // 2, lib=lib)
    S = np.zeros(nq)
    excluded = np.zeros(nq, dtype=bool)
    half = m // 2
    pad = int(np.floor((k_context - 1.0) * m / 2.0))
    elems, chosen = [], []
    smax = np.inf
    for it in range(max_elements):
        Pp = np.where(excluded, np.inf, P - S)
        finite = np.isfinite(Pp)
        if not finite.any():
            break
        j = int(np.argmin(np.where(finite, Pp, np.inf)))  # argmin: lowest index on ties
        chosen.append(j)
        elems.append((max(0, j - pad), min(n, j + m + pad)))
        excluded[max(0, j - half):min(nq, j + half)] = True
        Sp, _, _ = ab_join(x, x[j:j + m], np.array([0, m]), m, lib=lib)  # distance profile of window j
        S = Sp if it == 0 else np.minimum(S, Sp)
        smax = float(S.max())
        total = sum(b - a for a, b in _merge(elems))
        if term == "memory" and total >= term_value:
            break
        if term == "emax" and smax <= term_value:
            break
    segs = [(a, b - a) for a, b in _merge(elems)]
    return segs, chosen, smax


def _merge(iv):
    out = []
    for a, b in sorted(iv):
        if out and a < out[-1][1]:
            out[-1] = (out[-1][0], max(out[-1][1], b))
        else:
            out.append((a, b))
    return out

