"""The FP64 -> FP32/TF32 conversions the kernels build on the integer pipes,
and the FP64 Newton division of the FP64 energy epilogue, modelled on the
host operation for operation and checked against their definitions without a
GPU:

* TF32 from the high word of a double: round half away from zero to 10
  mantissa bits (the first dropped bit lies in the high word), magnitudes
  below 2^-126 to signed zero;
* FP32 from both words: round half away from zero to 23 mantissa bits, the
  same flush;
* FP64 from FP32: exact;
* v / x by Newton steps on the reciprocal from an FP32 seed, the last step
  folded into the product: one step within 2^-43 relative, two within a few
  FP64 roundings.
"""
import struct
from fractions import Fraction

import numpy as np


def _bits64(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _f32_of_bits(u):
    return struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0]


def tf32_from_f64_hi(hi):
    sign = hi & 0x80000000
    r = ((hi & 0x7FFFFFFF) + (1 << 9)) >> 10
    e = (r >> 10) - 896
    return _f32_of_bits(sign | ((r - (896 << 10)) << 13)) if e > 0 else _f32_of_bits(sign)


def f32_from_f64_bits(lo, hi):
    sign = hi & 0x80000000
    e = ((hi >> 20) & 0x7FF) - 896
    m = ((e << 23) | ((hi & 0xFFFFF) << 3) | (lo >> 29)) & 0xFFFFFFFF
    m += (lo >> 28) & 1
    return _f32_of_bits(sign | m) if e > 0 else _f32_of_bits(sign)


def _round_away(x, bits):
    """x rounded half away from zero to `bits` significant bits (exact)."""
    q = Fraction(float(x))
    if q == 0:
        return q
    s = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    unit = Fraction(2) ** (e - bits + 1)
    n = q / unit
    f = n.numerator // n.denominator
    if n - f >= Fraction(1, 2):
        f += 1
    return s * f * unit


def _doubles(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * 10.0 ** rng.uniform(-30, 30, n)
    # values on the rounding ties and just below a power of two (carry into the exponent)
    ties = [(1 + (2 * k + 1) * 2.0 ** -11) * 2.0 ** rng.integers(-60, 60) for k in range(50)]
    ties += [(1 + (2 * k + 1) * 2.0 ** -24) * 2.0 ** rng.integers(-60, 60) for k in range(50)]
    carry = [(2 - 2.0 ** -40) * 2.0 ** rng.integers(-60, 60) for _ in range(20)]
    v = np.concatenate([x, ties, carry, -np.array(ties), -np.array(carry)])
    return v


def test_tf32_and_fp32_from_fp64_bits():
    for x in _doubles(4000, seed=7):
        b = _bits64(x)
        hi, lo = b >> 32, b & 0xFFFFFFFF
        t = tf32_from_f64_hi(hi)
        f = f32_from_f64_bits(lo, hi)
        if abs(x) < 2.0 ** -126:
            assert t == 0.0 and f == 0.0
            continue
        assert Fraction(t) == _round_away(x, 11), x
        assert Fraction(f) == _round_away(x, 24), x
        assert np.float64(np.float32(f)) == f and (_bits64(t) & ((1 << 42) - 1)) == 0   # FP32 / TF32 values
    # flush to signed zero below 2^-126
    for x in (3e-39, -3e-39, 1e-300):
        b = _bits64(x)
        assert f32_from_f64_bits(b & 0xFFFFFFFF, b >> 32) == 0.0


def fma64(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def div_newton(v, x, steps):
    r = float(np.float32(1.0) / np.float32(x))          # the FP32 reciprocal seed, modelled as rounded
    for _ in range(steps - 1):
        r = fma64(r, fma64(-x, r, 1.0), r)
    e = fma64(-x, r, 1.0)
    t = v * r
    return fma64(t, e, t)


def test_newton_division_steps():
    rng = np.random.default_rng(8)
    worst = {1: 0.0, 2: 0.0}
    for _ in range(3000):
        x = -rng.uniform(0.05, 8.0)                    # e_i + e_j - e_a - e_b
        v = rng.standard_normal() * 10.0 ** rng.uniform(-6, -1)
        exact = Fraction(v) / Fraction(x)
        for s in (1, 2):
            worst[s] = max(worst[s], float(abs(Fraction(div_newton(v, x, s)) - exact) / abs(exact)))
    assert worst[1] <= 2.0 ** -43
    assert worst[2] <= 2.0 ** -51
