"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw 2011,
"Parallel random numbers: as easy as 1, 2, 3", SC11).

Every random number the sampler draws is a pure function of (counter, key), so
the CPU and the GPU walk draw identical streams without sharing state.  Pinned
against numpy.random.Philox, which implements the same published generator.
"""
import numpy as np

_MASK = (1 << 64) - 1
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B


def philox4x64(counter, key):
    """One 10-round Philox4x64 block: counter (4 x u64), key (2 x u64) -> 4 x u64 (Python ints)."""
    c0, c1, c2, c3 = (int(x) & _MASK for x in counter)
    k0, k1 = (int(x) & _MASK for x in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & _MASK, (p0 >> 64) ^ c3 ^ k1, p0 & _MASK)
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def mulhi(x: int, n: int) -> int:
    """floor(x * n / 2^64): an index uniform on [0, n) from a 64-bit draw."""
    return (int(x) * int(n)) >> 64


def open_unit(x: int) -> float:
    """Uniform double on (0, 1) from a 64-bit draw: ((x >> 12) + 1/2) / 2^52 (exact, never 0 or 1)."""
    return ((int(x) >> 12) + 0.5) * (1.0 / 4503599627370496.0)


def philox4x64_array(counters: np.ndarray, key) -> np.ndarray:
    """Vectorised Philox4x64-10 over rows of counters [n, 4] (uint64) -> [n, 4] uint64."""
    out = np.empty((counters.shape[0], 4), dtype=np.uint64)
    for i in range(counters.shape[0]):
        out[i] = philox4x64(counters[i], key)
    return out


_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.ndarray, b: np.uint64):
    """(high, low) 64-bit halves of the 128-bit products a * b, elementwise on uint64."""
    a_lo, a_hi = a & _M32, a >> _S32
    b_lo, b_hi = np.uint64(int(b) & 0xFFFFFFFF), np.uint64(int(b) >> 32)
    p0 = a_lo * b_lo
    p1 = a_lo * b_hi
    p2 = a_hi * b_lo
    p3 = a_hi * b_hi
    mid = (p0 >> _S32) + (p1 & _M32) + (p2 & _M32)
    hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    with np.errstate(over="ignore"):
        lo = a * b
    return hi, lo


def philox4x64_vec(c0, c1, c2, c3, key):
    """Philox4x64-10 on arrays of counter words (uint64, broadcastable) -> tuple of 4 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) for x in np.broadcast_arrays(c0, c1, c2, c3))
    k0, k1 = int(key[0]) & _MASK, int(key[1]) & _MASK
    for _ in range(10):
        hi0, lo0 = _mulhilo(c0, np.uint64(_M0))
        hi1, lo1 = _mulhilo(c2, np.uint64(_M1))
        c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def mulhi_vec(x: np.ndarray, n) -> np.ndarray:
    """floor(x * n / 2^64) elementwise (n < 2^32)."""
    hi, _ = _mulhilo(np.asarray(x, dtype=np.uint64), np.uint64(int(n)))
    return hi.astype(np.int64)


def open_unit_vec(x: np.ndarray) -> np.ndarray:
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(12)).astype(np.float64) + 0.5) * (1.0 / 4503599627370496.0)
