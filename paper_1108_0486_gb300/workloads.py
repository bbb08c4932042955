"""Seeded synthetic inputs of the benchmark and test workloads.

Holds none of the generator's arithmetic: only seeds, sizes and request
mixes, drawn with numpy's PCG64.  Shared by the tests (which feed the same
inputs to the GPU path and to the CPU oracle) and by bench.py.

The paper's own workload is "generate 10^8 random numbers repeatedly"
(Sec. 3); it has no dataset.  Streams are seeded with consecutive integers,
as the paper seeds each block with its block id (Sec. 4).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KIND_NAMES = ("u32", "uniform", "normal")


def seeds(n: int, start: int = 1) -> np.ndarray:
    """Consecutive seeds start, start+1, ... (block ids, Sec. 4)."""
    return np.arange(start, start + n, dtype=np.uint64).astype(np.uint32)


# single stream, 2^20 words, seed 0x12345678
SINGLE_STREAM = dict(seed=0x12345678, n=1 << 20)
# 16384 streams x 2^16 words (2^30 words = 4 GiB) of u32 plus as many uniforms
MANY_STREAMS = dict(streams=16384, n=1 << 16)
# 2^30 FP32 normals over 16384 streams
NORMALS = dict(streams=16384, n=1 << 16)


@dataclass
class BatchItem:
    stream: int
    kind: int      # 0 u32, 1 uniform, 2 normal
    count: int


def batched_uneven(n_streams: int = 4096, lo: int = 1 << 10, hi: int = 1 << 24,
                   seed: int = 1108):
    """One item per stream: lengths log-uniform in [lo, hi], kinds uniform over
    {u32, uniform, normal}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), n_streams))).astype(np.int64)
    lens = np.clip(lens, lo, hi)
    kinds = rng.integers(0, 3, n_streams)
    return [BatchItem(i, int(k), int(c)) for i, (k, c) in enumerate(zip(kinds, lens))]


@dataclass
class Request:
    t_arrival: float   # seconds from the start
    stream: int
    kind: int
    count: int


def serving_requests(n_streams: int = 65536, rate: float = 20000.0, duration: float = 10.0,
                     lo: int = 1 << 10, hi: int = 1 << 22, mix=(0.1, 0.3, 0.6), seed: int = 486):
    """Open-loop Poisson arrivals; sizes log-uniform in [lo, hi]; kinds drawn
    with probabilities mix = (u32, uniform, normal); streams uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_expected = int(rate * duration * 1.2) + 16
    gaps = rng.exponential(1.0 / rate, n_expected)
    t = np.cumsum(gaps)
    t = t[t < duration]
    m = t.size
    sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), m))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    kinds = rng.choice(3, size=m, p=np.asarray(mix) / np.sum(mix))
    streams = rng.integers(0, n_streams, m)
    return [Request(float(a), int(s), int(k), int(c)) for a, s, k, c in zip(t, streams, kinds, sizes)]
