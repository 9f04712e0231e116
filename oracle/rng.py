"""Counter-based N(0,1) generator for start and replacement blocks (Table 1, MvRandom).

SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a hash of (seed, stream, counter), then the
Box-Muller transform (Box & Muller 1958): z = sqrt(-2 ln(1 - u1)) cos(2 pi u2) with u1, u2
uniform on [0, 1) from the top 53 bits of two consecutive counters.  Element i of a block
uses counters 2i and 2i+1.  Test infrastructure only (the CUDA library has its own copy,
written from the same published definitions).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)
_OFFSET = np.uint64(0x632BE59BD9B4E019)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def sm64_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        s0 = _mix(np.array([np.uint64(seed) * _GOLDEN + np.uint64(stream) * _STREAM + _OFFSET],
                           dtype=np.uint64))[0]
        return _mix(s0 + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * _GOLDEN)


def uniform01(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    return (sm64_at(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal_block(n: int, b: int, seed: int, stream: int, offset: int = 0) -> np.ndarray:
    """Row-major n x b block of N(0,1) draws; element (r, c) has index offset + r*b + c."""
    i = np.arange(n * b, dtype=np.uint64) + np.uint64(offset)
    u1 = uniform01(seed, stream, 2 * i)
    u2 = uniform01(seed, stream, 2 * i + 1)
    return (np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)).reshape(n, b)
