"""The digit scheme of the BF16x2 tensor-core form (the headline mixed form),
modelled on the host with its integer and FP32 steps reproduced: the claims
its kernel and its GPU tolerances rest on, checked without a GPU.

The first half contracts a row chunk of 32 FP64 integrals x with a C_Y
column c (Eq. (dp2e), the p2 quarter transformation) on the tensor cores:

* x in 16-bit fixed point relative to the chunk's largest exponent field
  e_max: y = x 2^(15 - e), e = e_max - 1023, built from the high word of each
  double only (its 20 mantissa bits hold every bit above the rounding
  position), the lowest FP32 mantissa bit of y set to stand for the dropped
  low word; balanced digits d0 = rn(y / 2^8), d1 = rn(y - 2^8 d0), so that
  2^8 d0 + d1 = rn(y);
* c (FP32) in 32-bit fixed point relative to the column's largest exponent:
  four balanced base-256 digits of rn(c 2^(31 - f));
* the tensor cores sum the digit products by level, L0 = sum a0 b0,
  L1 = sum (a0 b1 + a1 b0), L2 = sum (a0 b2 + a1 b1), in FP32 -- exact while
  every partial sum stays below 2^24;
* T = 2^(e + f - 14) ((L2 2^-8 + L1) 2^-8 + L0), two FP32 FMAs.

Checked here: the digits of every element are the correctly rounded fixed
point of the full double (ties away from zero) and exact in BF16; every level
sum is below 2^24 for up to 128 p2 terms; and T is within the fixed point's
rounding bound of the exact sum.
"""
import struct
from fractions import Fraction

import numpy as np

from fp32_model import F32, Q, f32, fma

MAGIC = F32(12582912.0)   # 1.5 * 2^23: x + MAGIC - MAGIC rounds x to an integer


def _hi_word(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0] >> 32


def _as_f32(bits):
    return np.frombuffer(struct.pack("<I", bits & 0xFFFFFFFF), dtype=np.float32)[0]


def a_digits(xs):
    """The chunk's (emax, [(d0, d1)]) as the converter builds them."""
    his = [_hi_word(x) for x in xs]
    emax = max(h & 0x7FFFFFFF for h in his) >> 20
    K = (emax - 142) << 20
    out = []
    for h in his:
        t = max((h & 0x7FFFFFFF) - K, 0)
        y = _as_f32((t << 3) | 1 | (h & 0x80000000))
        d0 = f32(Q(fma(y, F32(2.0 ** -8), MAGIC)) - Q(MAGIC))
        r = fma(d0, F32(-256.0), y)
        assert Q(r) == Q(y) - 256 * Q(d0)           # the remainder is exact
        d1 = f32(Q(f32(Q(r) + Q(MAGIC))) - Q(MAGIC))
        out.append((d0, d1))
    return emax, out


def b_digits(cs):
    """C_Y column (FP32) as (f, [(b0, b1, b2, b3)]): 32-bit fixed point digits."""
    fmax = max(int(np.frombuffer(struct.pack("<f", float(c)), dtype=np.uint32)[0]) >> 23 & 0xFF for c in cs)
    scale = F32(2.0 ** (158 - fmax))
    out = []
    for c in cs:
        y = f32(Q(c) * Q(scale))
        d = []
        for s in (2.0 ** -24, 2.0 ** -16, 2.0 ** -8, 1.0):
            dk = f32(Q(fma(y, F32(s), MAGIC)) - Q(MAGIC))
            d.append(dk)
            y = fma(-dk, F32(1.0 / s), y)
        out.append(tuple(d))
    return fmax - 127, out


def _round_half_away(q):
    f = q.numerator // q.denominator
    rem = q - f
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q > 0):
        return f + 1
    return f


def _is_bf16(v):
    """v exactly representable in BF16 (8 significant bits)."""
    bits = int(np.frombuffer(struct.pack("<f", float(v)), dtype=np.uint32)[0])
    return bits & 0xFFFF == 0


def _chunks(n, seed):
    rng = np.random.default_rng(seed)
    for t in range(n):
        x = rng.standard_normal(32) * 10.0 ** rng.uniform(-9, 0, 32)
        if t % 4 == 0:                               # exact ties of the fixed point, both signs
            e = int(np.floor(np.log2(np.max(np.abs(x)))))
            for k in range(4):
                x[k] = (-1) ** k * (rng.integers(1, 2 ** 14) + 0.5) * 2.0 ** (e - 15)
        if t % 5 == 0:
            x[rng.integers(0, 32, 5)] = 0.0
        c = (rng.standard_normal(32) * 10.0 ** rng.uniform(-3, 0, 32)).astype(F32)
        yield x, c


def test_a_digits_are_the_rounded_fixed_point():
    for x, _ in _chunks(120, seed=1):
        emax, ds = a_digits(x)
        e = emax - 1023
        for xv, (d0, d1) in zip(x, ds):
            assert abs(d0) <= 256 and abs(d1) <= 128 and _is_bf16(d0) and _is_bf16(d1)
            z = Q(xv) * Fraction(2) ** (15 - e)      # the exact scaled value
            expected = _round_half_away(z) if z >= 0 else -_round_half_away(-z)
            assert 256 * Q(d0) + Q(d1) == expected, (xv, d0, d1, expected)


def test_b_digits_are_the_rounded_fixed_point():
    for _, c in _chunks(60, seed=2):
        f, ds = b_digits(c)
        for cv, d in zip(c, ds):
            assert abs(d[0]) <= 256 and all(abs(v) <= 128 for v in d[1:]) and all(_is_bf16(v) for v in d)
            y = Q(cv) * Fraction(2) ** (31 - f)
            got = sum(Q(dk) * 256 ** (3 - k) for k, dk in enumerate(d))
            assert abs(got - y) <= Fraction(1, 2)


def test_level_sums_exact_and_contraction_within_bound():
    worst = 0.0
    for x, c in _chunks(120, seed=3):
        emax, ad = a_digits(x)
        f, bd = b_digits(c)
        e = emax - 1023
        L = [sum(Q(a[0]) * Q(b[0]) for a, b in zip(ad, bd)),
             sum(Q(a[0]) * Q(b[1]) + Q(a[1]) * Q(b[0]) for a, b in zip(ad, bd)),
             sum(Q(a[0]) * Q(b[2]) + Q(a[1]) * Q(b[1]) for a, b in zip(ad, bd))]
        # every partial sum of 32 terms, and the bound for 128, below 2^24
        for lev in range(3):
            acc = Fraction(0)
            for a, b in zip(ad, bd):
                terms = [(0, 0)] if lev == 0 else [(0, 1), (1, 0)] if lev == 1 else [(0, 2), (1, 1)]
                for i, j in terms:
                    acc += Q(a[i]) * Q(b[j])
                    assert abs(acc) < 2 ** 24
        Lf = [f32(v) for v in L]
        assert all(Q(a) == b for a, b in zip(Lf, L))
        v = fma(fma(Lf[2], F32(2.0 ** -8), Lf[1]), F32(2.0 ** -8), Lf[0])
        T = Q(v) * Fraction(2) ** (e + f - 14)
        exact = sum(Q(a) * Q(b) for a, b in zip(x, c))
        # bound: half a unit of each element's fixed point times max|c|, 32 terms,
        # plus the dropped level and the two FP32 roundings of the combination
        scale = float(Fraction(2) ** e * max(abs(Q(cv)) for cv in c))
        err = abs(float(T - exact)) / scale
        worst = max(worst, err)
        assert err <= 32 * 2.0 ** -16 + 2.0 ** -20
    # worst-case digits: 128 terms of the largest level products stay exact
    assert 128 * (256 * 128 + 128 * 256) < 2 ** 24
    print(f"worst |T - sum x c| / (2^e max|c|) = 2^{np.log2(worst):.1f}")
