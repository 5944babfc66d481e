"""Counter-based splitmix64 streams (Steele, Lea & Flood, OOPSLA 2014).

Value i of stream (seed, tag) is mix64(seed + golden * (i + 1) + tag * 2^32-ish salt),
where mix64 is the splitmix64 output function.  Everything is vectorised with
numpy uint64 wraparound arithmetic, so a stream is reproducible bit for bit on any
machine and any numpy version.  This module holds no star-forest arithmetic.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Base seed for the five workload families: 0x5F2102130180000 + family number.
BASE_SEED = 0x5F2102130180000


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _salt(seed: int, tag: int) -> np.uint64:
    # Derive a per-(seed, tag) starting state; tag separates independent streams.
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        t = mix64(np.array([np.uint64(tag & 0xFFFFFFFFFFFFFFFF) ^ np.uint64(0xD1B54A32D192ED03)]))[0]
        return s ^ t


def u64(seed: int, tag: int, n: int, start: int = 0) -> np.ndarray:
    """n raw 64-bit values of stream (seed, tag), starting at counter `start`."""
    base = _salt(seed, tag)
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(base + GOLDEN * i)


def uniform01(seed: int, tag: int, n: int) -> np.ndarray:
    """Doubles uniform in [0, 1): top 53 bits times 2^-53 (exact)."""
    return (u64(seed, tag, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def randint(seed: int, tag: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi) by 64-bit multiply-high (Lemire), exact in uint64."""
    span = hi - lo
    if span <= 0:
        raise ValueError("empty range")
    x = u64(seed, tag, n)
    # multiply-high of x by span using 32-bit halves (no 128-bit type in numpy)
    span64 = np.uint64(span)
    xh = x >> np.uint64(32)
    xl = x & np.uint64(0xFFFFFFFF)
    sh = span64 >> np.uint64(32)
    sl = span64 & np.uint64(0xFFFFFFFF)
    with np.errstate(over="ignore"):
        ll = xl * sl
        lh = xl * sh
        hl = xh * sl
        hh = xh * sh
        mid = (ll >> np.uint64(32)) + (lh & np.uint64(0xFFFFFFFF)) + (hl & np.uint64(0xFFFFFFFF))
        hi64 = hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))
    return hi64.astype(np.int64) + lo
