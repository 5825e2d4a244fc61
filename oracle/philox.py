"""Philox4x32-10 and Box-Muller in vectorized numpy (oracle; test infrastructure only).

The Wigner noise of Sec. III.B.1 (Eq. sample) is drawn from a counter-based
generator so that the CUDA path and this oracle see the same random numbers
without sharing code.  Philox4x32-10 is written from its published definition
(J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with the round keys
bumped by the Weyl constants between rounds.

Counter layout used for the Wigner noise of cell g, stream slot s, instance i:
    ctr = (g, s, i, 0),  key = (seed mod 2^32, seed >> 32).
Of the four output words, x0 and x1 give the two uniforms of one Box-Muller pair.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds on uint32 counter arrays (broadcast), key (k0, k1).

    Returns four uint32 arrays.  Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by (W0, W1)
    before every round after the first.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    ka = int(k0) & 0xFFFFFFFF
    kb = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            ka = (ka + _W0) & 0xFFFFFFFF
            kb = (kb + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(ka)), lo1, (hi0 ^ c3 ^ np.uint64(kb)), lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def uniform_open(x) -> np.ndarray:
    """Map a uint32 word to the open interval (0, 1): u = (x + 1/2) / 2^32, in FP64."""
    return (np.asarray(x, dtype=np.float64) + 0.5) * (1.0 / 4294967296.0)


def box_muller(x0, x1):
    """Two independent N(0,1) variates from two uint32 words (Box & Muller 1958), FP64.

    r = sqrt(-2 ln u0), theta = 2 pi u1;  returns (r cos theta, r sin theta).
    """
    u0 = uniform_open(x0)
    u1 = uniform_open(x1)
    r = np.sqrt(-2.0 * np.log(u0))
    th = 2.0 * np.pi * u1
    return r * np.cos(th), r * np.sin(th)


def wigner_normals(seed: int, n_cells: int, slot: int, instance: int = 0):
    """Standard normal pair (zR, zI) for every cell of one stream slot (FP64 arrays)."""
    g = np.arange(n_cells, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(g, slot, instance, 0, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return box_muller(x0, x1)
