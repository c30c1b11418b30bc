"""Counter-based random streams built on SplitMix64.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) is used as a counter-based generator: output i of a
stream with key k is mix(k + (i + 1) * 0x9E3779B97F4A7C15), where mix is the
published SplitMix64 finaliser. Because every output depends only on (key, i),
the streams are reproducible bit for bit on any machine and any numpy version,
and they vectorise without a Python loop.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(key: int, start: int, n: int) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream whose state starts at `key`."""
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & _MASK64) + idx * _GOLDEN
    return _mix(z)


def _hash_tag(key: int, tag) -> int:
    """Derive a child key from a parent key and a tag (str or int)."""
    if isinstance(tag, str):
        h = 1469598103934665603  # FNV-1a 64 over the UTF-8 bytes
        for b in tag.encode():
            h = ((h ^ b) * 1099511628211) & _MASK64
        tag = h
    v = splitmix64((key ^ (int(tag) * 0xD6E8FEB86659FD93)) & _MASK64, 0, 1)[0]
    return int(v)


class Stream:
    """A named, seeded random stream. `child(tag)` gives an independent stream."""

    def __init__(self, seed: int, *path):
        key = int(seed) & _MASK64
        for tag in path:
            key = _hash_tag(key, tag)
        self.key = key
        self.pos = 0

    def child(self, *tags) -> "Stream":
        s = Stream.__new__(Stream)
        key = self.key
        for tag in tags:
            key = _hash_tag(key, tag)
        s.key = key
        s.pos = 0
        return s

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.key, self.pos, int(n))
        self.pos += int(n)
        return out

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits of each output."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform on [lo, hi) (hi > lo)."""
        span = int(hi) - int(lo)
        if span <= 0:
            raise ValueError("empty range")
        v = np.floor(self.uniform(n) * span).astype(np.int64)
        return np.minimum(v, span - 1) + int(lo)

    def log_uniform_int(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers with log-uniform distribution on [lo, hi]."""
        a, b = np.log(float(lo)), np.log(float(hi) + 1.0)
        v = np.floor(np.exp(a + (b - a) * self.uniform(n))).astype(np.int64)
        return np.clip(v, lo, hi)

    def scalar_uniform(self, lo: float, hi: float) -> float:
        return float(lo + (hi - lo) * self.uniform(1)[0])
