"""Pins of the reference codecs (oracle/quant.py) to the formats' definitions."""
import numpy as np

from oracle import quant


def test_bf16_known_points():
    x = np.array([1.0, -2.5, 0.0, 3.140625, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0], np.float32)
    b = quant.bf16_bits(x)
    assert b[0] == 0x3F80 and b[1] == 0xC020 and b[2] == 0
    assert b[3] == 0x4049                    # 3.140625 is exact in bf16
    assert b[4] == 0x3F80                    # tie at 1 + 2^-8 goes to the even mantissa
    assert b[5] == 0x3F82                    # tie at 1 + 3 * 2^-8 rounds up to even
    # bf16 -> fp32 -> bf16 is the identity on every finite pattern
    bits = np.arange(0, 0x7F80, 7, dtype=np.uint16)
    assert (quant.bf16_bits(quant.bf16_value(bits)) == bits).all()


def test_e4m3_table():
    v = quant._VALUES
    assert v[0x7E] == 448.0 and np.isnan(v[0x7F])     # S.1111.110 is the largest finite value
    assert v[0x01] == 2.0 ** -9                       # smallest subnormal
    assert v[0x08] == 2.0 ** -6                       # smallest normal
    assert v[0x38] == 1.0                             # exponent field 7 = bias
    finite = v[:0x7F]
    assert (np.diff(finite) > 0).all()                # codes 0..126 increase


def test_e4m3_rounding_brute_force():
    # every code round-trips; midpoints go to the even code; saturation at 448
    for c in range(0x7F):
        assert quant.e4m3_codes(np.array([quant._VALUES[c]], np.float32))[0] == c
        assert quant.e4m3_codes(np.array([-quant._VALUES[c]], np.float32))[0] == (c | 0x80 if c else 0)
    for c in range(0x7E):
        mid = (quant._VALUES[c] + quant._VALUES[c + 1]) / 2
        got = quant.e4m3_codes(np.array([mid], np.float32))[0]
        if np.float32(mid) == mid:
            assert got == (c if c % 2 == 0 else c + 1)
    assert quant.e4m3_codes(np.array([1e6, -1e6, 449.0], np.float32)).tolist() == [0x7E, 0xFE, 0x7E]


def test_fp8_row_scale():
    x = np.array([0.0, 1.0, -3.5, 7.0], np.float32)
    codes, s = quant.fp8_row(x)
    assert s == np.float32(7.0) / np.float32(448.0)
    assert quant._VALUES[codes[3]] == 448.0
    z, s0 = quant.fp8_row(np.zeros(5, np.float32))
    assert s0 == 1.0 and (z == 0).all()
