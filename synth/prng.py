"""SplitMix64 as a counter-based generator (numpy, vectorised).

Output i of a generator seeded with s is mix(s + (i + 1) * GAMMA), where mix is
the published SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014).
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the generator seeded with ``seed``."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA)


def at(seed, index) -> np.ndarray:
    """Output ``index`` (array) of generators seeded with ``seed`` (array)."""
    seed = np.asarray(seed, dtype=np.uint64)
    index = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix(seed + (index + np.uint64(1)) * GAMMA)


def derive(*parts: int) -> int:
    """A 64-bit seed derived from integers (for per-buffer / per-array seeds)."""
    s = 0x0DB0_5EED_0000_0001
    for p in parts:
        s = int(mix(np.uint64((s ^ (p & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF)))
    return s


class Rng:
    """Sequential draws from one SplitMix64 stream (host-side trace shaping)."""

    def __init__(self, seed: int):
        self.seed = seed & 0xFFFFFFFFFFFFFFFF
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = stream(self.seed, self.pos, n)
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers in [lo, hi) (hi - lo <= 2**32; multiply-shift reduction)."""
        span = np.uint64(hi - lo)
        x = self.u64(n) >> np.uint64(32)
        with np.errstate(over="ignore"):
            return (lo + ((x * span) >> np.uint64(32))).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        u1 = np.maximum(u1, 1e-300)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def permutation(self, n: int) -> np.ndarray:
        keys = self.u64(n)
        return np.argsort(keys, kind="stable")
