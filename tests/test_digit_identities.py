"""Integer identities the split slicer relies on, checked on the CPU.

The slicer (split.cu, split_common.cuh) cuts each FP64 value into balanced
base-2^beta digits with a few bit-level shortcuts. These tests check the
identities behind the shortcuts on plain Python integers (no GPU, no library):

* rounding half away from zero by one shift: (M + 2^(r-1)) >> r equals
  ((M >> (r-1)) + 1) >> 1 for r >= 1, and is 0 once r > 53 for M < 2^53;
* a BETA-bit field at bit o of a 32-bit word, gathered for two words with one
  byte permute of the 16-bit windows at byte b = min(o // 8, 2) and one shift,
  equals the two fields extracted separately whenever o - 8 b + BETA <= 16;
* the BF16 pattern 0x4300 + f is the value 128 + f for 0 <= f < 128, so one
  subtraction of 128 + 2^(BETA-1) gives the balanced digit f - 2^(BETA-1);
* the line exponent taken from the separate maxima of the two 32-bit halves
  of |x|, also after merging such pairs of several items as 64-bit values,
  equals the one taken from the 64-bit maximum.
"""
import random
import struct

import numpy as np


def _bf16_value(bits16):
    return struct.unpack("<f", struct.pack("<I", bits16 << 16))[0]


def _byte_perm(x, y, sel):
    b = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    return sum(b[(sel >> (4 * i)) & 7] << (8 * i) for i in range(4))


def _line_exponent(bits):
    if bits == 0:
        return 0
    eb = (bits >> 52) & 0x7FF
    if eb:
        return eb - 1022
    return (bits & ((1 << 52) - 1)).bit_length() - 1074


def test_round_half_away_by_one_shift():
    rnd = random.Random(1)
    for _ in range(20000):
        M = rnd.getrandbits(rnd.randint(1, 53))
        r = rnd.randint(1, 70)
        want = (M + (1 << (r - 1))) >> r
        got = ((M >> (r - 1)) + 1) >> 1 if r <= 53 else 0
        assert got == want, (M, r)


def test_byte_window_gathers_two_fields():
    rnd = random.Random(2)
    for beta in (6, 7):
        mask = (1 << beta) - 1
        for o in range(0, 32 - beta + 1):
            b = min(o // 8, 2)
            if o - 8 * b + beta > 16:
                continue
            sel = b | (b + 1) << 4 | (b + 4) << 8 | (b + 5) << 12
            for _ in range(300):
                w0, w1 = rnd.getrandbits(32), rnd.getrandbits(32)
                both = (_byte_perm(w0, w1, sel) >> (o - 8 * b)) & (mask * 0x10001)
                assert both & 0xFFFF == (w0 >> o) & mask
                assert both >> 16 == (w1 >> o) & mask


def test_bf16_small_integer_patterns():
    for beta in (6, 7):
        half = 1 << (beta - 1)
        sub = _bf16_value(0x4300 + half)
        assert sub == 128 + half
        for f in range(1 << beta):
            assert _bf16_value(0x4300 + f) == 128 + f
            # the packed subtraction is exact: the digit is representable
            d = np.float32(_bf16_value(0x4300 + f)) - np.float32(sub)
            assert d == f - half


def test_line_exponent_from_halves():
    rnd = random.Random(3)

    def bits(x):
        return struct.unpack("<Q", struct.pack("<d", x))[0] & ((1 << 63) - 1)

    for _ in range(3000):
        kind = rnd.random()
        if kind < 0.4:
            xs = [rnd.uniform(-1, 1) * 10.0 ** rnd.uniform(-300, 300) for _ in range(16)]
        elif kind < 0.8:
            xs = [struct.unpack("<d", struct.pack("<Q", rnd.getrandbits(rnd.randint(1, 52))))[0]
                  for _ in range(16)]
        else:
            xs = [0.0] * 15 + [5e-324 * rnd.randint(0, 1 << 20)]
        full = max(bits(x) for x in xs)
        hi = max(bits(x) >> 32 for x in xs)
        lo = max(bits(x) & 0xFFFFFFFF for x in xs)
        assert _line_exponent(hi << 32 | lo) == _line_exponent(full)
        # per-item pairs merged as 64-bit values (the shared-memory atomicMax)
        cut = rnd.randint(1, 15)
        pairs = [max(bits(x) >> 32 for x in part) << 32 | max(bits(x) & 0xFFFFFFFF for x in part)
                 for part in (xs[:cut], xs[cut:])]
        assert _line_exponent(max(pairs)) == _line_exponent(full)
