"""Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written from the published definition.

One call maps a 256-bit counter (four 64-bit words) and a 128-bit key to 256
random bits.  Round: two 64x64->128 multiplications by the Philox constants,
an xor with the round key and a word permutation; the key is bumped by the
Weyl constants between rounds; 10 rounds.

How the method consumes the stream (a reading the paper leaves open; it
only says Q is random, Sec. 5.2, and pivots are uniform, Sec. 5.1):

* JL matrix Q (k x m): key = (seed, TAG_JL); for edge id e and block
  c = i // 256 of JL rows, counter = (e, c, 0, 0).  Row i's sign is bit
  (i % 64) of output word (i % 256) // 64: bit 0 -> +1/sqrt(k), 1 -> -1/sqrt(k).
* Pivot sampling: key = (seed, TAG_SAMPLE); Floyd step j draws word 0 of
  counter (j, 0, 0, 0).

Pinned: ``tests/test_oracle_philox.py`` checks this function against numpy's
``np.random.Philox`` bit generator (also Philox4x64-10).
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B

TAG_JL = 0x4A4C  # "JL"
TAG_SAMPLE = 0x534D50  # "SMP"

_MASK64 = (1 << 64) - 1
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x64_10_int(ctr, key):
    """Scalar reference on Python integers: ctr is 4 words, key 2 words."""
    x = [int(c) & _MASK64 for c in ctr]
    k0, k1 = int(key[0]) & _MASK64, int(key[1]) & _MASK64
    for _ in range(10):
        p0 = M0 * x[0]
        p1 = M1 * x[2]
        x = [(p1 >> 64) ^ x[1] ^ k0, p1 & _MASK64, (p0 >> 64) ^ x[3] ^ k1, p0 & _MASK64]
        k0 = (k0 + W0) & _MASK64
        k1 = (k1 + W1) & _MASK64
    return x


def _mulhilo(a: np.ndarray, b: int):
    """64x64 -> (hi, lo) on uint64 arrays via 32-bit limbs."""
    b = np.uint64(b)
    a_lo = a & _LO32
    a_hi = a >> _S32
    b_lo = b & _LO32
    b_hi = b >> _S32
    t = a_lo * b_lo
    u = a_hi * b_lo + (t >> _S32)
    v = a_lo * b_hi + (u & _LO32)
    hi = a_hi * b_hi + (u >> _S32) + (v >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x64-10 over uint64 counter arrays (broadcast).
    Returns four uint64 arrays."""
    with np.errstate(over="ignore"):
        x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3))
        x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
        ka = np.uint64(k0 & _MASK64)
        kb = np.uint64(k1 & _MASK64)
        for _ in range(10):
            hi0, lo0 = _mulhilo(x0, M0)
            hi1, lo1 = _mulhilo(x2, M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ ka, lo1, hi0 ^ x3 ^ kb, lo0
            ka = ka + np.uint64(W0)
            kb = kb + np.uint64(W1)
    return x0, x1, x2, x3
