"""Python binding of libmpdict (include/mpdict.h): the dictionary AB-join on a GB300.

The functions carry the C ABI's names and only marshal arguments: every step of
the join runs in the library's CUDA kernels. There is no CPU fallback; if the
shared library has not been built, importing this package raises.

Host arrays are numpy arrays; device arrays are passed as raw pointers (for
example ``tensor.data_ptr()`` of a CUDA torch tensor) together with a stream
handle (``torch.cuda.current_stream().cuda_stream``) or 0 for the context's own
stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpdict.so")

MP_OK = 0
MP_E_ARG = -1
MP_E_NOMEM = -2
MP_E_CUDA = -3
MP_E_NOTFOUND = -4
MP_E_BUSY = -5
MP_E_TIMEOUT = -6
MP_E_INTERNAL = -7

MP_F32 = 0
MP_F64 = 1

MP_KERNEL_AUTO = 0
MP_KERNEL_PLAIN = 1
MP_KERNEL_TC_BF16X3 = 2
MP_KERNEL_TC_TF32 = 3
MP_KERNEL_TC_BF16 = 4

MP_PHASE_STATS = 0
MP_PHASE_JOIN = 1
MP_PHASE_FINALIZE = 2
MP_PHASE_SEEDS = 3
MP_PHASE_LEFT_SEEDS = 4
MP_PHASE_COUNT = 5

MP_COUNTER_NEAR_ROWS = 0
MP_COUNTER_NEAR_CHUNKS = 1
MP_COUNTER_OVERFLOW_ROWS = 2
MP_COUNTER_OVERFLOW_CHUNKS = 3
MP_COUNTER_COUNT = 4

MP_HOOK_FAIL_ALLOC = 0
MP_HOOK_TC_WAIT = 1

MP_LEARN_MEMORY = 0
MP_LEARN_EMAX = 1

MP_PENDING = 0
MP_DONE = 1
MP_FAILED = 2

_CODES = {
    MP_E_ARG: "MP_E_ARG",
    MP_E_NOMEM: "MP_E_NOMEM",
    MP_E_CUDA: "MP_E_CUDA",
    MP_E_NOTFOUND: "MP_E_NOTFOUND",
    MP_E_BUSY: "MP_E_BUSY",
    MP_E_TIMEOUT: "MP_E_TIMEOUT",
    MP_E_INTERNAL: "MP_E_INTERNAL",
}


class MPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class mp_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("max_inflight", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("mem_budget", ctypes.c_size_t),
        ("tune_cache", ctypes.c_char_p),
        ("max_pending", ctypes.c_int32),
    ]


class mp_join_plan(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("column_groups", ctypes.c_int32),
        ("spans", ctypes.c_int64),
        ("row_chunks", ctypes.c_int64),
        ("tc_seeds", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("workspace_bytes", ctypes.c_int64),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()'). "
            "There is no CPU fallback."
        )
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sig = {
        "mp_config_default": ([ctypes.POINTER(mp_config)], ctypes.c_int),
        "mp_init": ([ctypes.POINTER(P), ctypes.POINTER(mp_config)], ctypes.c_int),
        "mp_shutdown": ([P], ctypes.c_int),
        "mp_last_error": ([], ctypes.c_char_p),
        "mp_set_kernel": ([P, i32], ctypes.c_int),
        "mp_dict_load": ([P, P, i32, P, i32, P, i32, ctypes.POINTER(P)], ctypes.c_int),
        "mp_dict_free": ([P, P], ctypes.c_int),
        "mp_dict_windows": ([P, i32, ctypes.POINTER(i64)], ctypes.c_int),
        "mp_ab_join": ([P, P, P, i32, i64, i32, P, P], ctypes.c_int),
        "mp_ab_join_corr": ([P, P, P, i32, i64, i32, P, P], ctypes.c_int),
        "mp_stream_open": ([P, P, i32, i32, ctypes.POINTER(P)], ctypes.c_int),
        "mp_stream_append": ([P, P, i64, P, P, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "mp_stream_close": ([P], ctypes.c_int),
        "mp_stream_submit": ([P, P, i64, P, P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i64),
                              ctypes.POINTER(i64)], ctypes.c_int),
        "mp_self_join": ([P, P, i32, i64, i32, i32, P, P], ctypes.c_int),
        "mp_learn_dictionary": ([P, P, i32, i64, i32, ctypes.c_double, i32, ctypes.c_double, i32, P, P,
                                 ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(i32)],
                                ctypes.c_int),
        "mp_ab_join_device": ([P, P, P, i32, i64, i32, P, P, P], ctypes.c_int),
        "mp_ab_join_noalloc": ([P, P, P, i32, i64, i32, P, P, P], ctypes.c_int),
        "mp_window_stats": ([P, P, i32, i64, i32, P, P, P, P], ctypes.c_int),
        "mp_submit": ([P, P, P, i32, i64, i32, P, P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "mp_poll": ([P, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "mp_drain": ([P, ctypes.c_double], ctypes.c_int),
        "mp_profile": ([P, i32], ctypes.c_int),
        "mp_emax": ([P, P, P, i32, i64, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)], ctypes.c_int),
        "mp_top_discords": ([P, i64, i32, i64, ctypes.c_double, P, P, ctypes.POINTER(i32), ctypes.POINTER(i32)],
                            ctypes.c_int),
        "mp_autotune": ([P, P, i32, i64, ctypes.c_double, ctypes.POINTER(i32), ctypes.POINTER(i32),
                         ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "mp_profile_read": ([P, P, P, i32], ctypes.c_int),
        "mp_counters": ([P, P, i32], ctypes.c_int),
        "mp_test_hook": ([P, i32, i64], ctypes.c_int),
        "mp_plan_join": ([P, P, i32, i64, i32, ctypes.POINTER(mp_join_plan)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def mp_last_error() -> str:
    return lib.mp_last_error().decode()


def _check(rc: int) -> None:
    if rc != MP_OK:
        raise MPError(rc, mp_last_error())


def _dtype_of(x: np.ndarray) -> int:
    if x.dtype == np.float32:
        return MP_F32
    if x.dtype == np.float64:
        return MP_F64
    raise TypeError(f"samples must be float32 or float64, not {x.dtype}")


def _ptr(x: np.ndarray) -> int:
    return x.ctypes.data


def mp_config_default() -> mp_config:
    cfg = mp_config()
    _check(lib.mp_config_default(ctypes.byref(cfg)))
    return cfg


def mp_init(cfg: Optional[mp_config] = None, **overrides) -> ctypes.c_void_p:
    """Create a context. Keyword overrides set fields of the default config."""
    if cfg is None:
        cfg = mp_config_default()
    for k, v in overrides.items():
        setattr(cfg, k, v.encode() if isinstance(v, str) else v)
    ctx = ctypes.c_void_p()
    _check(lib.mp_init(ctypes.byref(ctx), ctypes.byref(cfg)))
    return ctx


def mp_shutdown(ctx) -> None:
    _check(lib.mp_shutdown(ctx))


def mp_set_kernel(ctx, kernel: int) -> None:
    _check(lib.mp_set_kernel(ctx, kernel))


def mp_dict_load(ctx, samples: np.ndarray, seg_offsets: Sequence[int], ms: Sequence[int] = ()) -> ctypes.c_void_p:
    """Upload a dictionary: samples (float32/float64) cut by seg_offsets (len = n_segments + 1)."""
    samples = np.ascontiguousarray(samples)
    dt = _dtype_of(samples)
    offs = np.ascontiguousarray(seg_offsets, dtype=np.int64)
    msa = np.ascontiguousarray(ms, dtype=np.int32)
    d = ctypes.c_void_p()
    _check(lib.mp_dict_load(ctx, _ptr(samples) if samples.size else None, dt, _ptr(offs), len(offs) - 1,
                            _ptr(msa) if msa.size else None, len(msa), ctypes.byref(d)))
    return d


def mp_dict_free(ctx, d) -> None:
    _check(lib.mp_dict_free(ctx, d))


def mp_dict_windows(d, m: int) -> int:
    w = ctypes.c_int64()
    _check(lib.mp_dict_windows(d, m, ctypes.byref(w)))
    return w.value


def mp_ab_join(ctx, d, query: np.ndarray, m: int) -> Tuple[np.ndarray, np.ndarray]:
    """Synchronous join with host buffers; returns (distance, index) arrays of length n - m + 1."""
    q = np.ascontiguousarray(query)
    nq = max(len(q) - m + 1, 0)
    dist = np.empty(nq, dtype=np.float64)
    idx = np.empty(nq, dtype=np.int64)
    _check(lib.mp_ab_join(ctx, d, _ptr(q), _dtype_of(q), len(q), m, _ptr(dist), _ptr(idx)))
    return dist, idx


def mp_ab_join_corr(ctx, d, query: np.ndarray, m: int) -> Tuple[np.ndarray, np.ndarray]:
    """The join reported as correlation rho = 1 - d^2/(2m) (the largest per row); returns (rho, index)."""
    q = np.ascontiguousarray(query)
    nq = max(len(q) - m + 1, 0)
    corr = np.empty(nq, dtype=np.float64)
    idx = np.empty(nq, dtype=np.int64)
    _check(lib.mp_ab_join_corr(ctx, d, _ptr(q), _dtype_of(q), len(q), m, _ptr(corr), _ptr(idx)))
    return corr, idx


def mp_self_join(ctx, series: np.ndarray, m: int, excl: int) -> Tuple[np.ndarray, np.ndarray]:
    """Self-join matrix profile (float32): nearest window with |g - i| >= excl; returns (distance, index)."""
    x = np.ascontiguousarray(series)
    nq = max(len(x) - m + 1, 0)
    dist = np.empty(nq, dtype=np.float64)
    idx = np.empty(nq, dtype=np.int64)
    _check(lib.mp_self_join(ctx, _ptr(x), _dtype_of(x), len(x), m, excl, _ptr(dist), _ptr(idx)))
    return dist, idx


def mp_learn_dictionary(ctx, t_b: np.ndarray, m: int, k_context: float = 1.5, term: int = MP_LEARN_MEMORY,
                        term_value: float = 0.0, max_elements: int = 4096):
    """Algorithm 1 on the GPU; returns (segments [(start, length)], chosen windows, error bound max S)."""
    x = np.ascontiguousarray(t_b)
    starts = np.empty(max_elements, dtype=np.int64)
    lens = np.empty(max_elements, dtype=np.int64)
    chosen = np.empty(max_elements, dtype=np.int64)
    nseg = ctypes.c_int32()
    nch = ctypes.c_int32()
    bound = ctypes.c_double()
    _check(lib.mp_learn_dictionary(ctx, _ptr(x), _dtype_of(x), len(x), m, k_context, term, term_value, max_elements,
                                   _ptr(starts), _ptr(lens), ctypes.byref(nseg), ctypes.byref(bound),
                                   _ptr(chosen), ctypes.byref(nch)))
    segs = [(int(a), int(b)) for a, b in zip(starts[: nseg.value], lens[: nseg.value])]
    return segs, [int(c) for c in chosen[: nch.value]], bound.value


def mp_stream_open(ctx, d, dtype: int, m: int):
    """A streaming join of windows of length m against dictionary d; returns the stream handle."""
    h = ctypes.c_void_p()
    _check(lib.mp_stream_open(ctx, d, dtype, m, ctypes.byref(h)))
    return h


def mp_stream_append(stream, samples: np.ndarray) -> Tuple[np.ndarray, np.ndarray, int]:
    """Append samples; returns (distance, index, first window) of the windows that end in them."""
    x = np.ascontiguousarray(samples)
    n = len(x)
    dist = np.empty(max(n, 1), dtype=np.float64)
    idx = np.empty(max(n, 1), dtype=np.int64)
    n_out = ctypes.c_int64()
    first = ctypes.c_int64()
    _check(lib.mp_stream_append(stream, _ptr(x) if n else None, n, _ptr(dist), _ptr(idx), ctypes.byref(n_out),
                                ctypes.byref(first)))
    k = n_out.value
    return dist[:k].copy(), idx[:k].copy(), first.value


def mp_stream_submit(stream, samples: np.ndarray, out_dist: np.ndarray, out_idx: np.ndarray) -> Tuple[int, int, int]:
    """Append samples without waiting; returns (ticket or 0, windows, first window). The outputs (float64 /
    int64, at least len(samples) long) must stay alive until mp_poll reports the ticket done."""
    x = np.ascontiguousarray(samples)
    n = len(x)
    assert out_dist.dtype == np.float64 and out_idx.dtype == np.int64 and len(out_dist) >= n and len(out_idx) >= n
    t = ctypes.c_uint64()
    n_out = ctypes.c_int64()
    first = ctypes.c_int64()
    _check(lib.mp_stream_submit(stream, _ptr(x) if n else None, n, _ptr(out_dist), _ptr(out_idx), ctypes.byref(t),
                                ctypes.byref(n_out), ctypes.byref(first)))
    return t.value, n_out.value, first.value


def mp_stream_close(stream) -> None:
    _check(lib.mp_stream_close(stream))


def mp_ab_join_device(ctx, d, d_query: int, dtype: int, n: int, m: int, d_dist: int, d_idx: int,
                      stream: int = 0) -> None:
    """Join on device pointers, enqueued on `stream` (0: the context's stream)."""
    _check(lib.mp_ab_join_device(ctx, d, d_query, dtype, n, m, d_dist, d_idx, stream or None))


def mp_ab_join_noalloc(ctx, d, d_query: int, dtype: int, n: int, m: int, d_dist: int, d_idx: int,
                       stream: int = 0) -> None:
    """Join on device pointers using the library's fixed scratch array (no device allocation)."""
    _check(lib.mp_ab_join_noalloc(ctx, d, d_query, dtype, n, m, d_dist, d_idx, stream or None))


def mp_window_stats(ctx, d_x: int, dtype: int, n: int, m: int, d_mean: int, d_invstd: int, d_const: int,
                    stream: int = 0) -> None:
    _check(lib.mp_window_stats(ctx, d_x, dtype, n, m, d_mean, d_invstd, d_const, stream or None))


def mp_submit(ctx, d, query: np.ndarray, m: int, out_dist: np.ndarray, out_idx: np.ndarray) -> int:
    """Queue a request; out_dist / out_idx (length n - m + 1) must stay alive until it is done."""
    q = np.ascontiguousarray(query)
    nq = len(q) - m + 1
    assert out_dist.dtype == np.float64 and out_idx.dtype == np.int64
    assert out_dist.flags.c_contiguous and out_idx.flags.c_contiguous
    assert len(out_dist) >= nq and len(out_idx) >= nq
    t = ctypes.c_uint64()
    _check(lib.mp_submit(ctx, d, _ptr(q), _dtype_of(q), len(q), m, _ptr(out_dist), _ptr(out_idx), ctypes.byref(t)))
    return t.value


def mp_poll(ctx, ticket: int) -> Tuple[int, float]:
    st = ctypes.c_int32()
    lat = ctypes.c_double(-1.0)
    _check(lib.mp_poll(ctx, ticket, ctypes.byref(st), ctypes.byref(lat)))
    return st.value, lat.value


def mp_drain(ctx, timeout_s: float = 60.0) -> None:
    _check(lib.mp_drain(ctx, timeout_s))


def mp_profile(ctx, enable: bool) -> None:
    _check(lib.mp_profile(ctx, 1 if enable else 0))


def mp_profile_read(ctx, reset: bool = False) -> Tuple[np.ndarray, np.ndarray]:
    """Per-phase device milliseconds and launch counts recorded since the last reset."""
    ms = np.zeros(MP_PHASE_COUNT, dtype=np.float64)
    n = np.zeros(MP_PHASE_COUNT, dtype=np.int64)
    _check(lib.mp_profile_read(ctx, _ptr(ms), _ptr(n), 1 if reset else 0))
    return ms, n


def mp_plan_join(ctx, d, dtype: int, n: int, m: int) -> dict:
    """The plan mp_ab_join_device would run for n query samples at window length m."""
    p = mp_join_plan()
    _check(lib.mp_plan_join(ctx, d, dtype, n, m, ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in mp_join_plan._fields_ if k != "pad"}


def mp_counters(ctx, reset: bool = False) -> np.ndarray:
    """Finalisation counters (MP_COUNTER_*) summed over the context's joins since the last reset."""
    v = np.zeros(MP_COUNTER_COUNT, dtype=np.int64)
    _check(lib.mp_counters(ctx, _ptr(v), 1 if reset else 0))
    return v


def mp_test_hook(ctx, hook: int, value: int) -> None:
    """Host-side fault injection for tests (MP_HOOK_*)."""
    _check(lib.mp_test_hook(ctx, hook, value))


def mp_autotune(ctx, d, m: int, n: int, tolerance: float = 1e-4) -> Tuple[int, int, float]:
    """Time the join forms for (dictionary, m, query length n); returns (kernel, groups, ms) of the fastest."""
    k = ctypes.c_int32()
    g = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(lib.mp_autotune(ctx, d, m, n, tolerance, ctypes.byref(k), ctypes.byref(g), ctypes.byref(ms)))
    return k.value, g.value, ms.value


def mp_emax(ctx, d, t_b: np.ndarray, m: int) -> Tuple[float, int]:
    """e_max of the dictionary for the series t_b it was learned from: (value, window attaining it)."""
    x = np.ascontiguousarray(t_b)
    e = ctypes.c_double()
    a = ctypes.c_int64()
    _check(lib.mp_emax(ctx, d, _ptr(x), _dtype_of(x), len(x), m, ctypes.byref(e), ctypes.byref(a)))
    return e.value, a.value


def mp_top_discords(profile: np.ndarray, k: int, excl: int, e_max: float = -1.0):
    """Top-k discords of a profile with a +-excl exclusion zone; returns (idx, val, top1_certified)."""
    pr = np.ascontiguousarray(profile, dtype=np.float64)
    idx = np.empty(max(k, 1), dtype=np.int64)
    val = np.empty(max(k, 1), dtype=np.float64)
    nf = ctypes.c_int32()
    cert = ctypes.c_int32()
    _check(lib.mp_top_discords(_ptr(pr), len(pr), k, excl, e_max, _ptr(idx), _ptr(val), ctypes.byref(nf),
                               ctypes.byref(cert)))
    return idx[: nf.value], val[: nf.value], bool(cert.value)
