"""Seeded generators for the synthetic stand-ins of the paper's data.

The paper evaluates on MIT-BIH Long-Term ECG (Sec. 4.4), on a surgery ECG
(Sec. 4.5) and on the Melbourne Pedestrian counts (Sec. 4.1), and its Fig. 1
uses random and random-walk series. None of those datasets is available here,
so each is replaced by a generator with the same kind of structure:

* ``random_walk``    -- cumulative sum of N(0, 1) steps, as in Fig. 1.
* ``ecg_like``       -- quasi-periodic heartbeats built from five Gaussian bumps
                        (P, Q, R, S, T waves) with period and amplitude jitter,
                        white noise, and optional malformed (PVC-like) beats
                        that play the role of the annotated anomalies of Sec. 4.4.
* ``transport_like`` -- 288 samples per day, daily and weekly sinusoids with a
                        per-day amplitude, Poisson spikes and white noise, standing
                        in for the pedestrian counts of Sec. 4.1.

Every generator takes an explicit seed and draws from
``numpy.random.default_rng(seed)``, so both sides of a comparison see identical
samples. Only input recipes live here; nothing in this module computes window
statistics, distances or minima.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# waveforms
# ---------------------------------------------------------------------------


def random_walk(n: int, seed: int) -> np.ndarray:
    """Random walk of ``n`` samples: cumulative sum of standard normal steps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal(n))


# Gaussian bumps of one heartbeat: (amplitude, centre, width), centre and width
# as fractions of the beat period.
_NORMAL_BEAT = (
    (+0.15, 0.20, 0.025),  # P wave
    (-0.10, 0.36, 0.008),  # Q
    (+1.00, 0.40, 0.010),  # R
    (-0.20, 0.44, 0.010),  # S
    (+0.30, 0.65, 0.040),  # T wave
)
# Malformed (PVC-like) beat: no P wave, a wide negative complex, larger T.
_MALFORMED_BEAT = (
    (-0.10, 0.36, 0.008),
    (-0.60, 0.42, 0.040),
    (-0.20, 0.44, 0.010),
    (+0.50, 0.70, 0.060),
)


def ecg_like(
    n: int,
    seed: int,
    n_malformed: int = 0,
    period: int = 180,
    period_jitter: float = 0.10,
    amp_jitter: float = 0.05,
    noise: float = 0.02,
    return_beats: bool = False,
):
    """ECG-like series of ``n`` samples.

    Beats follow each other without gaps. Beat ``b`` has a period drawn from
    ``period * U(1 - period_jitter, 1 + period_jitter)`` (rounded to whole
    samples) and an amplitude factor from ``U(1 - amp_jitter, 1 + amp_jitter)``.
    ``n_malformed`` beats, chosen uniformly without replacement among the beats
    that surely fit in the series, use the malformed template. White noise
    N(0, noise^2) is added to every sample.

    With ``return_beats`` the function also returns ``(starts, malformed)``:
    the start sample of every beat and a boolean mask of the malformed ones.
    """
    rng = np.random.default_rng(seed)
    max_period = int(np.ceil(period * (1 + period_jitter)))
    n_beats = n // int(np.floor(period * (1 - period_jitter))) + 2
    periods = np.rint(period * rng.uniform(1 - period_jitter, 1 + period_jitter, n_beats)).astype(np.int64)
    amps = rng.uniform(1 - amp_jitter, 1 + amp_jitter, n_beats)
    starts = np.concatenate(([0], np.cumsum(periods)[:-1]))
    malformed = np.zeros(n_beats, dtype=bool)
    if n_malformed > 0:
        fit = max(1, n // max_period - 1)  # beats that certainly lie inside [0, n)
        if n_malformed > fit:
            raise ValueError("too many malformed beats for the series length")
        malformed[rng.choice(fit, size=n_malformed, replace=False)] = True

    t = np.arange(n, dtype=np.int64)
    beat = np.searchsorted(starts, t, side="right") - 1
    phase = (t - starts[beat]) / periods[beat]
    x = np.zeros(n, dtype=np.float64)
    for amp, centre, width in _NORMAL_BEAT:
        x += np.where(~malformed[beat], amp * np.exp(-0.5 * ((phase - centre) / width) ** 2), 0.0)
    for amp, centre, width in _MALFORMED_BEAT:
        x += np.where(malformed[beat], amp * np.exp(-0.5 * ((phase - centre) / width) ** 2), 0.0)
    x *= amps[beat]
    x += rng.normal(0.0, noise, n)
    if return_beats:
        last = int(beat[-1]) + 1
        return x, (starts[:last], malformed[:last])
    return x


def transport_like(n: int, seed: int, day: int = 288, noise: float = 0.1) -> np.ndarray:
    """Transportation-like series: ``day`` samples per day.

    ``a_d * sin(2 pi t / day) + 0.5 * sin(2 pi t / (7 day))`` with a per-day
    amplitude ``a_d ~ U(0.8, 1.2)``, Poisson spikes (one per two days on
    average, height Exp(mean 2), 1 to 3 samples wide) and N(0, noise^2) noise.
    """
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64)
    n_days = n // day + 1
    a_d = rng.uniform(0.8, 1.2, n_days)
    x = a_d[(np.arange(n) // day)] * np.sin(2 * np.pi * t / day) + 0.5 * np.sin(2 * np.pi * t / (7 * day))
    n_spikes = rng.poisson(n / (2 * day))
    pos = rng.integers(0, n, n_spikes)
    height = rng.exponential(2.0, n_spikes)
    width = rng.integers(1, 4, n_spikes)
    for p, h, w in zip(pos, height, width):
        x[p : p + w] += h
    x += rng.normal(0.0, noise, n)
    return x


def cut_dictionary(series: np.ndarray, n_segments: int, seg_len: int) -> Tuple[np.ndarray, np.ndarray]:
    """Cut ``n_segments`` segments of ``seg_len`` samples at evenly spaced starts.

    Segment ``s`` starts at ``s * (len(series) // n_segments)``. Returns the
    concatenated samples and the ``int64`` offsets array of length
    ``n_segments + 1`` (segment ``s`` is ``samples[offsets[s]:offsets[s+1]]``).
    Because every segment is a contiguous piece of ``series``, every window of
    the dictionary is also a window of the series (Proposition 1).
    """
    stride = len(series) // n_segments
    if stride < seg_len:
        raise ValueError("segments would overlap")
    parts = [series[s * stride : s * stride + seg_len] for s in range(n_segments)]
    offsets = np.arange(n_segments + 1, dtype=np.int64) * seg_len
    return np.concatenate(parts), offsets


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------


@dataclass
class Workload:
    """One join problem: query, dictionary segments and window length."""

    name: str
    query: np.ndarray
    dict_samples: np.ndarray
    offsets: np.ndarray
    m: int
    dtype: str  # "f64" or "f32": the sample type handed to the join
    notes: dict = field(default_factory=dict)

    @property
    def n_rows(self) -> int:
        return max(0, len(self.query) - self.m + 1)

    @property
    def n_dict_windows(self) -> int:
        lens = np.diff(self.offsets)
        return int(np.maximum(lens - self.m + 1, 0).sum())

    @property
    def pairs(self) -> int:
        return self.n_rows * self.n_dict_windows


def _as(dtype: str, x: np.ndarray) -> np.ndarray:
    return x.astype(np.float32 if dtype == "f32" else np.float64)


def workload(name: str, scale: float = 1.0) -> Workload:
    """Build a named workload.

    ``scale`` < 1 shrinks the query (and, for the large cases, the training
    series) for quick tests while keeping the window length, segment length
    and generator; ``scale=1`` is the full size.

    Names:
      ``rw_fp64_4k``     random walk query of 4096 (seed 0), 8 x 256 dictionary
                         cut from an 8192 walk (seed 1), m = 64, float64.
      ``ecg_1m_m256``    ECG-like query of 2^20 (seed 2, 20 malformed beats),
                         64 x 1024 dictionary cut from a 2^20 series (seed 3),
                         m = 256, float32 samples.
      ``transport_4m_m512`` transportation-like query of 2^22 (seed 4),
                         256 x 2048 dictionary from a seed-5 series, m = 512.
      ``ecg_16m_m1024_dict`` / ``ecg_16m_m1024_orig`` ECG-like query of 2^24
                         (seed 7, 200 malformed beats) against a 128 x 2048
                         dictionary cut from a normal-beat 2^22 training series
                         (seed 6), or against that whole training series as one
                         segment; m = 1024.
    """
    def n_(x: int) -> int:
        return max(int(x * scale), 1)

    if name == "rw_fp64_4k":
        q = random_walk(n_(4096), 0)
        b, offs = cut_dictionary(random_walk(8192, 1), 8, 256)
        return Workload(name, _as("f64", q), _as("f64", b), offs, 64, "f64")
    if name == "ecg_1m_m256":
        nq = n_(1 << 20)
        q = ecg_like(nq, 2, n_malformed=min(20, max(1, nq // 200 - 1)))
        b, offs = cut_dictionary(ecg_like(1 << 20, 3), 64, 1024)
        return Workload(name, _as("f32", q), _as("f32", b), offs, 256, "f32")
    if name == "transport_4m_m512":
        q = transport_like(n_(1 << 22), 4)
        b, offs = cut_dictionary(transport_like(1 << 22, 5), 256, 2048)
        return Workload(name, _as("f32", q), _as("f32", b), offs, 512, "f32")
    if name in ("ecg_16m_m1024_dict", "ecg_16m_m1024_orig"):
        nq = n_(1 << 24)
        q = ecg_like(nq, 7, n_malformed=min(200, max(1, nq // 200 - 1)))
        train = ecg_like(n_(1 << 22), 6)
        if name.endswith("dict"):
            b, offs = cut_dictionary(train, 128, 2048)
        else:
            b, offs = train, np.array([0, len(train)], dtype=np.int64)
        return Workload(name, _as("f32", q), _as("f32", b), offs, 1024, "f32")
    raise KeyError(name)


WORKLOADS = ("rw_fp64_4k", "ecg_1m_m256", "transport_4m_m512", "ecg_16m_m1024_dict", "ecg_16m_m1024_orig")


# ---------------------------------------------------------------------------
# serving mix
# ---------------------------------------------------------------------------


@dataclass
class ServingRequest:
    arrival_s: float
    dict_id: int
    query: np.ndarray
    m: int


def serving_dictionaries(n_dicts: int = 16, seed: int = 100, min_log2: int = 14, max_log2: int = 18):
    """Resident dictionaries for the serving mix.

    Dictionary ``k`` has ``2^U`` samples in total, ``U ~ U{min_log2..max_log2}``,
    cut into segments whose lengths are uniform in [512, 4096] (the last one
    takes the remainder); its samples come from a random walk or an ECG-like
    series, alternating with ``k``.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_dicts):
        total = 1 << int(rng.integers(min_log2, max_log2 + 1))
        lens = []
        left = total
        while left > 0:
            L = int(rng.integers(512, 4097))
            L = min(L, left)
            lens.append(L)
            left -= L
        src = random_walk(total, seed + 1 + k) if k % 2 == 0 else ecg_like(total, seed + 1 + k)
        offs = np.concatenate(([0], np.cumsum(lens))).astype(np.int64)
        out.append((src.astype(np.float32), offs))
    return out


def serving_requests(
    n_requests: int = 10000,
    rate_hz: float = 100.0,
    seed: int = 200,
    n_dicts: int = 16,
    min_log2: int = 10,
    max_log2: int = 20,
    ms=(64, 128, 256),
) -> List[ServingRequest]:
    """Poisson arrivals of join requests.

    Inter-arrival times are Exp(1/rate_hz). Query length is ``2^U`` with
    ``U ~ U(min_log2, max_log2)`` (continuous, so lengths are log-uniform),
    the query is a random walk or an ECG-like series with probability 1/2 each,
    ``m`` is uniform over ``ms`` and the dictionary uniform over ``n_dicts``.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        n = int(2 ** rng.uniform(min_log2, max_log2))
        m = int(rng.choice(ms))
        n = max(n, m)
        s = int(rng.integers(0, 2**31 - 1))
        q = random_walk(n, s) if rng.random() < 0.5 else ecg_like(n, s)
        reqs.append(ServingRequest(t, int(rng.integers(0, n_dicts)), q.astype(np.float32), m))
    return reqs
