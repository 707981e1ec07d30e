"""FP8-E4M3 storage codec of A with a power-of-two scale per 128 x 128 tile (FP64 / numpy).

TEST INFRASTRUCTURE ONLY.  The codec is not part of the paper (which stores A in double
precision); it follows the reduced-precision storage the method is run with here:
    A~ = decode(q) * s_t,  q = E4M3(A / s_t) (round to nearest, ties to even, saturate to
    +-448),  s_t = 2^ceil(log2(max|A_t| / 448)) for every 128 x 128 tile t (s_t = 1 when the
    tile is zero).
E4M3 is written out from its definition: 1 sign bit, 4 exponent bits with bias 7, 3
mantissa bits; exponent field 0 holds the subnormals m * 2^-9; no infinities; the codes
S.1111.111 are NaN, so the largest finite magnitude is 1.75 * 2^8 = 448.
"""
from __future__ import annotations

import math

import numpy as np

TILE = 128
MAX_E4M3 = 448.0


def decode_e4m3(code: int) -> float:
    """Value of one E4M3 code (0..255)."""
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return math.nan
    if e == 0:
        return s * m * 2.0 ** -9
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def table() -> np.ndarray:
    return np.array([decode_e4m3(c) for c in range(256)])


_TAB = table()
# non-negative finite codes sorted by value (codes 0x00..0x7E increase monotonically)
_POS_CODES = np.arange(0x7F)
_POS_VALS = _TAB[:0x7F]


def encode_e4m3(x: np.ndarray) -> np.ndarray:
    """Round to the nearest E4M3 value (ties to the even code), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), MAX_E4M3)
    hi = np.clip(np.searchsorted(_POS_VALS, a, side="left"), 0, len(_POS_VALS) - 1)
    lo = np.maximum(hi - 1, 0)
    dlo = a - _POS_VALS[lo]
    dhi = _POS_VALS[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (_POS_CODES[hi] % 2 == 0))
    code = np.where(pick_hi, _POS_CODES[hi], _POS_CODES[lo]).astype(np.uint8)
    neg = (x < 0) & (code != 0)
    return np.where(neg, code | 0x80, code).astype(np.uint8)


def tile_scales(A: np.ndarray, tile: int = TILE) -> np.ndarray:
    """Power-of-two scale per tile: the smallest 2^k with max|A_t| / 2^k <= 448."""
    n0, n1 = A.shape
    nt0, nt1 = -(-n0 // tile), -(-n1 // tile)
    S = np.ones((nt0, nt1))
    for i in range(nt0):
        for j in range(nt1):
            m = float(np.max(np.abs(A[i * tile:(i + 1) * tile, j * tile:(j + 1) * tile])))
            if m > 0.0:
                k = math.ceil(math.log2(m / MAX_E4M3))
                while m / 2.0 ** k > MAX_E4M3:   # guard against log2 rounding
                    k += 1
                while k > -1074 and m / 2.0 ** (k - 1) <= MAX_E4M3:
                    k -= 1
                S[i, j] = 2.0 ** k
    return S


def quantize(A: np.ndarray, tile: int = TILE):
    """Returns (codes uint8 n0 x n1, scales per tile, A~ = decoded codes times scales)."""
    A = np.asarray(A, dtype=np.float64)
    S = tile_scales(A, tile)
    Sfull = np.repeat(np.repeat(S, tile, 0), tile, 1)[:A.shape[0], :A.shape[1]]
    codes = encode_e4m3(A / Sfull)
    return codes, S, _TAB[codes] * Sfull
