"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the solver. It only turns (seed, index) into numbers:

* ``splitmix64(seed, idx)`` -- the SplitMix64 mixing function (Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014), evaluated as a
  counter-based generator: output ``idx`` is the mix of the state ``seed + (idx + 1) * GOLDEN`` (the generator
  seeded with ``seed`` and advanced idx + 1 times).
* ``uniform_pm1(n, seed)`` -- n doubles uniform on [-1, 1), from the top 53 bits.
* ``problem(...)`` -- plain descriptions of the 1-D peridynamic problems of the paper's
  workloads (mesh size h = 2^-K, horizon delta, variant), with no matrix content.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counters ``idx`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(n: int, seed: int) -> np.ndarray:
    """n float64 values uniform on [-1, 1): 2 * (top 53 bits / 2^53) - 1."""
    if n == 0:
        return np.zeros(0, dtype=np.float64)
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


SPD = 0
NONSYM = 1


def problem(K: int, delta: float, variant: int = SPD) -> dict:
    """Description of the 1-D problem on (0,1) with N = 2^K intervals.

    Returns the mesh size h, the number of unknowns 2N - 1 (nodes then midpoints) and the
    requested horizon. The horizon ratio and every matrix entry are computed by the code
    that consumes this description, not here.
    """
    N = 1 << K
    return {"K": K, "N": N, "h": 1.0 / N, "delta": float(delta), "variant": int(variant),
            "n": 2 * N - 1}


# Workload families (sizes, horizons, variants) used by the tests and the benchmark.
SMALL_CASE = problem(7, 0.125, SPD)          # N = 128, delta = 1/8 (r = 16), 255 unknowns
LARGE_CASE = problem(22, 0.05, SPD)          # N = 2^22, delta = 0.05, 8,388,607 unknowns
