"""Seeded synthetic particle sets (inputs only).

This package draws the particle positions and masses that both the CUDA
path and the CPU oracle consume.  It holds no step of the tree build: no
quantisation, no key, no sort, no moment.  Every generator draws FP64
values from numpy's PCG64 stream (O'Neill 2014) for a given seed and
rounds them to FP32 once, at the end.

The per-step jitter of the batched workload is a counter-based draw
(SplitMix64 finaliser, Steele, Lea & Flood 2014) keyed by
(seed, step, set, particle, axis), so that any single value can be
reproduced without replaying a stream.
"""
from .generators import (  # noqa: F401
    uniform_cube,
    plummer,
    clustered_halos,
    precision_stress,
    exponential_disk,
    batched_plummer,
    jitter_offsets,
    splitmix64,
    lattice,
    workload,
    WORKLOADS,
)
