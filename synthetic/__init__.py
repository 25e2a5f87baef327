"""Seeded synthetic time series shaped like the paper's workloads.

This package is shared by the CPU oracle's tests and by the GPU path's tests
and benchmark. It holds input recipes only: random draws, waveform shapes and
the cutting of a dictionary from a training series. None of the join's
arithmetic (window statistics, distances, minima) lives here.
"""
from .generators import (  # noqa: F401
    random_walk,
    ecg_like,
    transport_like,
    cut_dictionary,
    Workload,
    workload,
    WORKLOADS,
    serving_requests,
    serving_dictionaries,
    ServingRequest,
)
