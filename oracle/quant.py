"""Reference codecs for the reduced-precision search copies.

TEST INFRASTRUCTURE (see oracle/etale_oracle.c for the rule on who may use it).

Written from the formats' definitions, not from any library conversion:
- bfloat16: the upper 16 bits of an IEEE binary32 after round-to-nearest,
  ties to even, of the lower 16 bits.
- FP8 E4M3 (OCP 8-bit floating point, E4M3 variant): 1 sign bit, 4 exponent
  bits with bias 7, 3 mantissa bits; exponent field 0 encodes subnormals
  (value m / 8 * 2^-6); S.1111.111 is NaN, so the largest finite value is
  S.1111.110 = 448.  Conversion rounds to nearest, ties to the even code;
  values beyond 448 saturate to +-448 (the "saturate to finite" mode).
- Per-vector scale of the FP8 copy: s = max|x| / 448 in fp32 (s = 1 for a
  zero row); codes encode x / s in fp32.
"""
from __future__ import annotations

import numpy as np


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even bf16 bits (uint16) of finite float32 values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    return ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)


def bf16_value(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def e4m3_value(code: int) -> float:
    """Exact value of an E4M3 code (NaN for S.1111.111)."""
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return s * (m / 8.0) * 2.0 ** -6
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


_CODES = np.arange(256)
_VALUES = np.array([e4m3_value(int(c)) for c in _CODES])


def e4m3_codes(v: np.ndarray) -> np.ndarray:
    """E4M3 codes of float32 values: nearest finite code, ties to the even
    code (even mantissa), saturating at +-448."""
    v = np.asarray(v, dtype=np.float32).astype(np.float64).ravel()
    finite = ~np.isnan(_VALUES)
    pos = (_CODES < 0x80) & finite
    pv, pc = _VALUES[pos], _CODES[pos]             # 0 .. 448 ascending
    order = np.argsort(pv)
    pv, pc = pv[order], pc[order]
    a = np.minimum(np.abs(v), 448.0)
    hi = np.clip(np.searchsorted(pv, a, side="left"), 0, len(pv) - 1)
    lo = np.clip(hi - 1, 0, len(pv) - 1)
    dlo, dhi = a - pv[lo], pv[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((pc[hi] & 1) == 0))
    code = np.where(pick_hi, pc[hi], pc[lo])
    code = np.where(a == pv[hi], pc[hi], code)
    neg = (v < 0) & (code != 0)
    return np.where(neg, code | 0x80, code).astype(np.uint8)


def fp8_row(x: np.ndarray) -> tuple[np.ndarray, np.float32]:
    """(codes, scale) of one row under the per-vector scale max|x| / 448."""
    x = np.asarray(x, dtype=np.float32)
    amax = np.float32(np.max(np.abs(x))) if x.size else np.float32(0)
    s = np.float32(amax / np.float32(448.0))
    if not s > 0:
        s = np.float32(1.0)
    return e4m3_codes((x / s).astype(np.float32)), s
