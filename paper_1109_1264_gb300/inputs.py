"""Seeded synthetic inputs for the SALT workloads.

This module holds no arithmetic of the method itself: it only draws the
operand vectors, scalars, lengths and request streams that both the CUDA
path and the CPU oracle are fed.  It imports nothing from either.

Workloads (all synthetic; the paper's own benchmarks are synthetic size
sweeps of xDOT, xSCAL, xAXPY and an out-of-place scaling, Section 5):

* ``uniform_vectors``: i.i.d. uniform[-1, 1] from ``numpy.random.default_rng``,
  drawn in FP64 in argument order, cast to FP32 when asked.
* ``logmag_vectors``: cancellation-heavy data, random sign times a magnitude
  log-uniform in [1e-3, 1e3].
* ``loguniform_lengths``: integer lengths log-uniform in [lo, hi].
* ``splitmix64`` / ``hash_uniform``: the counter-based generator that the
  device-side fill kernel also implements, so multi-GB batched inputs need no
  upload.  Element i of the stream keyed by ``key`` is output i+1 of
  SplitMix64 started from state ``key`` (Steele, Lea and Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014):
  ``z = key + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64), then the mix
  ``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
  z ^= z >> 31``.  FP64 value: ``2 * (z >> 11) * 2^-53 - 1``; FP32 value:
  ``2 * (z >> 40) * 2^-24 - 1``; both are exact in their format and lie in
  [-1, 1).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def uniform_vectors(seed: int, n: int, count: int, dtype=np.float64) -> list[np.ndarray]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        v = rng.uniform(-1.0, 1.0, n)
        out.append(np.ascontiguousarray(v.astype(dtype)))
    return out


def logmag_vectors(seed: int, n: int, count: int, dtype=np.float32,
                   lo_exp: float = -3.0, hi_exp: float = 3.0) -> list[np.ndarray]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
        mag = 10.0 ** rng.uniform(lo_exp, hi_exp, n)
        out.append(np.ascontiguousarray((sign * mag).astype(dtype)))
    return out


def loguniform_lengths(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = np.exp(rng.uniform(math.log(lo), math.log(hi), count))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def splitmix64(key: int, idx: np.ndarray) -> np.ndarray:
    """Output ``idx + 1`` of SplitMix64 started from state ``key``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def hash_uniform(key: int, n: int, dtype=np.float64, offset: int = 0) -> np.ndarray:
    """Elements ``offset .. offset+n-1`` of the keyed uniform[-1, 1) stream."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    h = splitmix64(key, idx)
    if dtype == np.float64:
        u = (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return 2.0 * u - 1.0
    u = (h >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return (2.0 * u - 1.0).astype(np.float32)


def vector_key(seed: int, item: int, slot: int) -> int:
    """Stream key of operand ``slot`` of work item ``item`` (distinct per pair)."""
    return (seed * 0x100000001B3 + item * 16 + slot + 1) & 0xFFFFFFFFFFFFFFFF


def cg_scalars(seed: int, count: int) -> np.ndarray:
    """(alpha, beta) per CG-style item, uniform(-1, 1)."""
    rng = np.random.default_rng(seed + 1)
    return rng.uniform(-1.0, 1.0, (count, 2))


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


def request_mix(seed: int, count: int, lo: int = 2 ** 8, hi: int = 2 ** 24,
                n_shapes: int = 5, f32_share: float = 0.7):
    """Served request stream: (shape index, is_fp64, n) per request."""
    rng = np.random.default_rng(seed)
    shapes = rng.integers(0, n_shapes, count)
    is64 = rng.random(count) >= f32_share
    lens = np.clip(np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))), lo, hi).astype(np.int64)
    return shapes, is64, lens
