"""Host checks of the arithmetic shortcuts the split kernels take in place of
FP64 division, against exact rational arithmetic (Python's Fraction; a float
made from a Fraction is correctly rounded).  The oracle computes a centroid
as the FP64 mean of FP32 values rounded to FP32 (Sec. 3.1's two-means); the
GPU must reach the same FP32 value.

1. Integer sums (data that an exact narrow copy holds): a sum S and a count K
   both exact in FP32 are divided in FP32, correctly rounded: RN32(S / K).
   The oracle's value is RN32(RN64(S / K)).  They agree: with S below 2^24
   the quotient is never an FP32 midpoint unless K divides it to a dyadic
   value FP64 holds exactly, and otherwise it lies farther from one than
   FP64's rounding error (K < 2^28).
2. FP64 sums: q0 = RN(s * inv) with inv = RN(1 / K), the residual
   r = RN(s - q0 K) (exact, as an FMA computes it) and q = RN(q0 + r inv)
   give RN(s / K) for integer s (Markstein's correction).
3. An unsigned byte b becomes the float 2^23 + b by placing it in the low
   mantissa bits of 2^23; subtracting 2^23 leaves b exactly.
"""
import random
import struct
from fractions import Fraction as F

import numpy as np


def rn64(x):
    return float(x)


def _rn32_frac(q):
    # correctly rounded FP32 of a rational: round to FP64 cannot be used
    # (double rounding), so round by hand from the exact value
    if q == 0:
        return np.float32(0.0)
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    # scale so that the significand has 24 bits before the point
    while F(2) ** e > q:
        e -= 1
    while F(2) ** (e + 1) <= q:
        e += 1
    scaled = q / F(2) ** (e - 23)          # in [2^23, 2^24)
    fl = scaled.numerator // scaled.denominator
    rem = scaled - fl
    if rem > F(1, 2) or (rem == F(1, 2) and fl % 2 == 1):
        fl += 1
    return np.float32(sign * float(F(fl) * F(2) ** (e - 23)))


def test_integer_mean_fp32_division_equals_fp64_then_fp32():
    rng = random.Random(5)
    cases = [(rng.randint(-(2**24) + 1, 2**24 - 1), rng.randint(1, 2**24 - 1)) for _ in range(20000)]
    cases += [(rng.randint(0, 2**24 - 1), rng.randint(1, 64)) for _ in range(20000)]
    # quotients just off FP32 midpoints: (2m + 1) / 2 scaled, perturbed by 1 / K
    cases += [(K * (2 * m + 1) // 2 + d, K) for m in range(2**22, 2**22 + 400) for K in (3, 7, 1023)
              for d in (-1, 0, 1) if K * (2 * m + 1) // 2 + d < 2**24]
    for S, K in cases:
        gpu = np.float32(S) / np.float32(K)                     # IEEE FP32 division
        oracle = np.float32(rn64(F(S, K)))                      # RN32(RN64(S / K))
        assert gpu == oracle, (S, K)
        assert gpu == _rn32_frac(F(S, K)), (S, K)               # both are RN32 of the exact quotient


def test_markstein_corrected_quotient_is_fp64_division():
    rng = random.Random(7)
    for _ in range(50000):
        K = rng.choice([rng.randint(1, 2**22), rng.randint(1, 64), 2**rng.randint(1, 22) - 1])
        s = rng.choice([rng.randint(0, 2**40), K * rng.randint(0, 2**20), K * rng.randint(0, 2**20) + 1])
        s = -s if rng.random() < 0.3 else s
        inv = rn64(F(1, K))
        q0 = rn64(F(s) * F(inv))
        r = rn64(F(s) - F(q0) * K)
        assert F(r) == F(s) - F(q0) * K            # the residual is exact
        q = rn64(F(q0) + F(r) * F(inv))
        assert q == rn64(F(s, K)), (s, K)


def test_byte_to_float_by_mantissa_placement():
    for b in range(256):
        bits = 0x4B000000 | b
        f = struct.unpack("<f", struct.pack("<I", bits))[0]
        assert f == 8388608.0 + b
        assert np.float32(f) - np.float32(8388608.0) == np.float32(b)
