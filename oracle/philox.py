"""Philox4x32-10 counter-based generator (oracle side).

TEST INFRASTRUCTURE ONLY.

Written from its published definition: J. K. Salmon, M. A. Moraes, R. O. Dror and
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11 (Philox with
four 32-bit words, two multipliers, Weyl key schedule, 10 rounds).  The random
numbers of the LAI sketch (the Gaussian test matrix of Sec. 2.3) and of the
default initialisation (Sec. 4.1, guideline (4)) are drawn from this generator
on both the oracle and the CUDA side, each with its own implementation.

Stream layout (shared by both implementations):
* Gaussian matrix, n x l row-major, flat index t: pair p = t // 2 uses
  counter (p mod 2^32, p div 2^32, 0, 0) and key (seed mod 2^32, seed div 2^32);
  u1 = (x0 + 1/2) 2^-32, u2 = (x1 + 1/2) 2^-32, z = sqrt(-2 ln u1) * cos(2 pi u2)
  for even t and * sin(2 pi u2) for odd t (Box-Muller).
* Uniform matrix, flat index t: counter (t mod 2^32, t div 2^32, 1, 0), same key,
  u = (x0 + 1/2) 2^-32.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Philox4x32 block function on arrays of 32-bit words (held in uint64)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for _ in range(rounds):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def _key(seed: int):
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(s & 0xFFFFFFFF), np.uint64(s >> 32)


def philox_gaussian(n: int, cols: int, seed: int) -> np.ndarray:
    """n x cols standard normal matrix from the Gaussian stream layout above."""
    total = n * cols
    npairs = (total + 1) // 2
    p = np.arange(npairs, dtype=np.uint64)
    k0, k1 = _key(seed)
    x0, x1, _, _ = philox4x32(p & _MASK, p >> _S32, 0, 0, k0, k1)
    u1 = (x0.astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (x1.astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:total].reshape(n, cols)


def philox_uniform(n: int, cols: int, seed: int) -> np.ndarray:
    """n x cols matrix of U(0,1) values from the uniform stream layout above."""
    t = np.arange(n * cols, dtype=np.uint64)
    k0, k1 = _key(seed)
    x0, _, _, _ = philox4x32(t & _MASK, t >> _S32, 1, 0, k0, k1)
    return ((x0.astype(np.float64) + 0.5) * 2.0 ** -32).reshape(n, cols)
