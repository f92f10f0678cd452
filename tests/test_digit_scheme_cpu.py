"""The arithmetic identities the FP64-class digit split relies on, checked on a host model (no GPU).

The split kernel cuts each value x of a row with largest biased exponent e_row into the fixed-point
integer X = round(x / 2^(e_row - 1061)), |X| <= 2^39, and reads its five signed base-256 digits
from the bytes of U = X + 0x8080808080 (128 in every digit position).  Each digit becomes a BF16
number through binary32 arithmetic: 2^23 + byte is exact, the subtraction of 2^23 + 128 is exact,
and so is the scaling by 2^p.  This file checks on random and edge values that
  * the digits reproduce X exactly, with d_1..d_4 in [-128, 127] and d_0 in [-128, 128];
  * the binary32 construction gives the same BF16 bits as building them from the integer digit
    (sign, exponent, fraction) for every digit and every row exponent of the fast range.
"""
import struct

import numpy as np

OFFSET = 0x8080808080


def fixed_point(v: float, eb_row: int) -> int:
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    eb = (b >> 52) & 0x7FF
    if eb == 0:
        return 0
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    rs = eb_row - eb + 14
    x = (m + (1 << (rs - 1))) >> rs if rs < 64 else 0
    return -x if b >> 63 else x


def byte_digits(x: int):
    u = x + OFFSET
    assert u >= 0
    lo = u & 0xFFFFFFFF
    return [(u >> 32) - 128] + [((lo >> (32 - 8 * s)) & 0xFF) - 128 for s in (1, 2, 3, 4)], u


def bf16_from_integer(d: int, p: int) -> int:
    if d == 0:
        return 0
    a = abs(d)
    msb = a.bit_length() - 1
    be = msb + p + 127
    if be <= 0:
        return 0
    sign = 0x8000 if d < 0 else 0
    if be >= 255:
        return sign | 0x7F80
    return sign | (be << 7) | ((a << (7 - msb)) & 0x7F)


def bf16_from_binary32(byte: int, p: int) -> int:
    f32 = lambda u: np.frombuffer(struct.pack("<I", u), dtype=np.float32)[0]
    with np.errstate(over="ignore"):
        f = (f32(0x4B000000 | byte) - np.float32(8388736.0)) * f32((p + 127) << 23)
    return struct.unpack("<I", struct.pack("<f", float(f)))[0] >> 16


def _values():
    rng = np.random.default_rng(7)
    vals = list(rng.normal(size=3000) * 10.0 ** rng.integers(-30, 30, 3000))
    return vals + [1.0, -1.0, 0.5, 2.0 ** 39, -(2.0 ** 39), 1 - 2 ** -53, -(1 - 2 ** -53), 127.5, 128.0, 0.0]


def test_byte_digits_reproduce_the_fixed_point_integer():
    for v in _values():
        e = (struct.unpack("<Q", struct.pack("<d", abs(v) if v else 1.0))[0] >> 52) & 0x7FF
        for eb_row in (e, e + 1, e + 9, e + 20):
            x = fixed_point(v, eb_row)
            d, _ = byte_digits(x)
            assert sum(di << (32 - 8 * s) for s, di in enumerate(d)) == x
            assert -128 <= d[0] <= 128 and all(-128 <= di <= 127 for di in d[1:])
            # the top digit is 128 exactly when X + offset reaches 2^40 (X within 2^31 of 2^39)
            assert (d[0] == 128) == (x >= (1 << 40) - OFFSET)


def test_binary32_construction_gives_the_integer_bf16_bits():
    for v in _values()[::3]:
        e = (struct.unpack("<Q", struct.pack("<d", abs(v) if v else 1.0))[0] >> 52) & 0x7FF
        for eb_row in (e, e + 3):
            if not 935 <= eb_row <= 1156:   # the kernel's fast range: every 2^p a normal binary32
                continue
            d, u = byte_digits(fixed_point(v, eb_row))
            for s in range(5):
                p = eb_row - 1029 - 8 * s
                byte = (u >> 32) if s == 0 else ((u & 0xFFFFFFFF) >> (32 - 8 * s)) & 0xFF
                assert bf16_from_binary32(byte, p) == bf16_from_integer(d[s], p), (v, eb_row, s)
