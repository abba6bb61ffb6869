"""E4M3 copies of training matrices with power-of-two scales (test
infrastructure).

The paper has no FP8; the library's FP8 training Gram (a stretch of the
training side, Section 3.1's Gram G = sum_d A_d A_d^T computed from 8-bit
copies) stores each training matrix in the E4M3 format with one
power-of-two scale per row and per group of eight consecutive matrices.  This
module restates that encoding from the format's definition, in float64 numpy:

* E4M3: 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits.  Exponent
  field E = 0 holds subnormals M * 2^-9; E in 1..15 holds (1 + M/8) 2^(E-7),
  except E = 15, M = 7, which is NaN.  There is no infinity; the largest
  finite magnitude is 448 (E = 15, M = 6).
* Rounding to E4M3 is to the nearest finite value, ties to the even code
  (even M), and magnitudes above 448 saturate to 448; the sign is kept
  (a negative value that rounds to zero gives the code 0x80).
* The scale of row i of group g is, for t = max over the group's matrices
  and the row's columns of |A_d[i, j]|, the smallest power of two
  s >= 2^-149 (FP32's smallest positive value) with t <= 448 s; s = 1 where
  t = 0.  Every stored byte is E4M3(A_d[i, j] / s) of the exact quotient.

The Gram of the copies, sum_d D_s A8_d A8_d^T D_s, is gram_mode1 of the
dequantised matrices.
"""
from __future__ import annotations

import numpy as np

GROUP = 8       # matrices per scale group
E4M3_MAX = 448.0


def e4m3_decode(codes) -> np.ndarray:
    """Values of E4M3 codes (uint8 array-like), from the format definition."""
    c = np.asarray(codes, dtype=np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    E = (c >> 3) & 0xF
    M = (c & 0x7).astype(np.float64)
    mag = np.where(E == 0, M * 2.0 ** -9, (1.0 + M / 8.0) * np.exp2(E - 7.0))
    mag = np.where((E == 15) & ((c & 7) == 7), np.nan, mag)
    return sign * mag


# the 127 finite non-negative values, in code order (codes 0x00..0x7E), which
# is also increasing order
_POS_CODES = np.arange(0x7F, dtype=np.int64)
_POS_VALUES = e4m3_decode(_POS_CODES)


def e4m3_encode(x) -> np.ndarray:
    """E4M3 codes (uint8) of finite float64 values: nearest finite value,
    ties to the even code, magnitudes above 448 saturated, sign kept."""
    x = np.asarray(x, dtype=np.float64)
    if not np.all(np.isfinite(x)):
        raise ValueError("e4m3_encode takes finite values")
    a = np.minimum(np.abs(x), E4M3_MAX)
    hi = np.clip(np.searchsorted(_POS_VALUES, a, side="left"), 0, len(_POS_VALUES) - 1)
    lo = np.maximum(hi - 1, 0)
    dlo = a - _POS_VALUES[lo]
    dhi = _POS_VALUES[hi] - a
    # nearer neighbour; on a tie the even code
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    mag = np.where(pick_hi, hi, lo)
    return (mag | np.where(np.signbit(x), 0x80, 0)).astype(np.uint8)


def row_scale(t) -> np.ndarray:
    """Scales for row maxima t >= 0: the smallest power of two s >= 2^-149
    with t <= 448 s, and 1 for t = 0 (float64; every value is exact)."""
    t = np.asarray(t, dtype=np.float64)
    es = np.zeros(t.shape, dtype=np.int64)
    pos = t > 0
    # a first guess from the logarithm, then exact corrections: 448 * 2^es
    # is exact in float64 over the whole range used
    g = np.ceil(np.log2(np.where(pos, t, 1.0) / E4M3_MAX)).astype(np.int64)
    g = np.maximum(g, -149)
    while True:
        up = pos & (t > E4M3_MAX * np.exp2(g.astype(np.float64)))
        if not up.any():
            break
        g = np.where(up, g + 1, g)
    while True:
        down = pos & (g > -149) & (t <= E4M3_MAX * np.exp2((g - 1).astype(np.float64)))
        if not down.any():
            break
        g = np.where(down, g - 1, g)
    es = np.where(pos, g, 0)
    return np.exp2(es.astype(np.float64))


def quantize_e4m3(As):
    """E4M3 copies and scales of D matrices (m x n each): returns (codes,
    scales) with codes a (D, m, n) uint8 array and scales (ceil(D / 8), m),
    scales[g, i] the scale of row i over matrices 8g .. 8g + 7."""
    A = np.stack([np.asarray(a, dtype=np.float64) for a in As])
    D, m, n = A.shape
    ng = (D + GROUP - 1) // GROUP
    scales = np.ones((ng, m))
    codes = np.zeros((D, m, n), dtype=np.uint8)
    for g in range(ng):
        blk = A[GROUP * g:GROUP * g + GROUP]
        t = np.abs(blk).max(axis=(0, 2)) if n > 0 else np.zeros(m)
        s = row_scale(t)
        scales[g] = s
        codes[GROUP * g:GROUP * g + GROUP] = e4m3_encode(blk / s[None, :, None])
    return codes, scales


def dequantize_e4m3(codes, scales) -> np.ndarray:
    """The values the copies stand for: decode(codes[d]) * scales[d // 8] per row."""
    codes = np.asarray(codes)
    D = codes.shape[0]
    s = np.asarray(scales, dtype=np.float64)[np.arange(D) // GROUP]
    return e4m3_decode(codes) * s[:, :, None]
