"""The digit scheme of the BF16x3 tensor-core form (the accurate mixed form),
modelled on the host with its integer and FP32 steps reproduced and checked
against exact rational arithmetic without a GPU.

The first half contracts a row chunk of 32 FP64 integrals x with a C_Y
column c (Eq. (dp2e), the p2 quarter transformation):

* x in 32-bit fixed point relative to the chunk's largest exponent field
  e_max: y = x 2^(31 - e), e = e_max - 1023, as FP32 built from the bit
  fields on the integer pipes -- the double's exponent and leading 23
  mantissa bits shifted into FP32 position, the exponent rebased by adding
  (158 - e_max) modulo 2^9, the first dropped mantissa bit added to the
  last kept one (rounding half away from zero), the sign put back; elements
  more than 2^157 below the largest become 0;
* four balanced base-256 digits of the integer nearest to y, each exact in
  BF16; c likewise in 32-bit fixed point relative to its column;
* level sums L_k = sum_{u+v=k} a_u b_v for k = 0..3 in FP32, exact while the
  partial sums stay below 2^24;
* T = 2^(e + f - 14) (((L3 2^-8 + L2) 2^-8 + L1) 2^-8 + L0), three FP32 FMAs.

y keeps the double's leading 24 significant bits, so the digits carry the
element to 24 significant bits, or to the unit of the 32-bit fixed point
where that is coarser.  Checked: every element's digits within |y| 2^-24 +
1/2 units of its exact fixed point (the 24-bit rounding of y, then the
integer rounding of the digits), level sums exact, and a chunk's contraction
within 2^-23 sum|x c| + 2^-26 2^e max|c| of the exact sum.
"""
import struct
from fractions import Fraction

import numpy as np

from fp32_model import F32, Q, f32, fma

MAGIC = F32(12582912.0)   # 1.5 * 2^23


def _bits64(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _as_f32(bits):
    return np.frombuffer(struct.pack("<I", bits & 0xFFFFFFFF), dtype=np.float32)[0]


def fx_y(x, emax):
    """y = x 2^(31 - e) as the converter forms it from the FP64 bit fields."""
    b = _bits64(x)
    hi, lo = b >> 32, b & 0xFFFFFFFF
    add = ((158 - emax) & 511) << 23
    thr = max(1, emax - 157) << 20
    w = ((((hi << 3) | (lo >> 29)) & 0xFFFFFFFF) + add + ((lo >> 28) & 1)) & 0xFFFFFFFF
    w = (w & 0x7FFFFFFF) | (hi & 0x80000000)
    return F32(0.0) if (hi & 0x7FFFFFFF) < thr else _as_f32(w)


def digits4(y):
    """Balanced base-256 digits of y (|y| < 2^32), as the converter's FMAs form them."""
    d = []
    for s in (2.0 ** -24, 2.0 ** -16, 2.0 ** -8, 1.0):
        dk = f32(Q(fma(y, F32(s), MAGIC)) - Q(MAGIC))
        d.append(dk)
        y = fma(-dk, F32(1.0 / s), y)
    return d


def _is_bf16(v):
    bits = int(np.frombuffer(struct.pack("<f", float(v)), dtype=np.uint32)[0])
    return bits & 0xFFFF == 0


def _value(d):
    return sum(Q(dk) * 256 ** (3 - k) for k, dk in enumerate(d))


def _chunks(n, seed):
    rng = np.random.default_rng(seed)
    for t in range(n):
        x = rng.standard_normal(32) * 10.0 ** rng.uniform(-12, 0, 32)
        if t % 5 == 0:
            x[rng.integers(0, 32, 5)] = 0.0
        c = (rng.standard_normal(32) * 10.0 ** rng.uniform(-3, 0, 32)).astype(F32)
        yield x, c


def _row_digits(x):
    emax = max(_bits64(v) >> 52 & 0x7FF for v in x)
    return emax, [digits4(fx_y(v, emax)) for v in x]


def test_row_digits_carry_24_significant_bits():
    worst_small = Fraction(0)
    for x, _ in _chunks(120, seed=4):
        emax, ds = _row_digits(x)
        e = emax - 1023
        for xv, d in zip(x, ds):
            assert abs(d[0]) <= 256 and all(abs(v) <= 128 for v in d[1:]) and all(_is_bf16(v) for v in d)
            y = Q(xv) * Fraction(2) ** (31 - e)
            err = abs(_value(d) - y)
            assert err <= abs(y) / 2 ** 24 + Fraction(1, 2), (xv, d)
            if abs(y) < 2 ** 23:
                worst_small = max(worst_small, err)
    # below 2^23 the integer rounding dominates: at most 3/4 of a unit
    assert worst_small <= Fraction(3, 4)
    print(f"worst digit error below 2^23: {float(worst_small):.3f} units")


def test_levels_exact_and_contraction_within_bound():
    worst = 0.0
    for x, c in _chunks(120, seed=5):
        emax, ad = _row_digits(x)
        e = emax - 1023
        fmax = max(int(np.frombuffer(struct.pack("<f", float(cv)), dtype=np.uint32)[0]) >> 23 & 0xFF for cv in c)
        f = fmax - 127
        bd = [digits4(f32(Q(cv) * Fraction(2) ** (158 - fmax))) for cv in c]
        L = []
        for k in range(4):
            acc = Fraction(0)
            for a, b in zip(ad, bd):
                for u in range(max(0, k - 3), min(k, 3) + 1):
                    acc += Q(a[u]) * Q(b[k - u])
                    assert abs(acc) < 2 ** 24
            L.append(acc)
        Lf = [f32(v) for v in L]
        assert all(Q(a) == b for a, b in zip(Lf, L))
        v = Lf[3]
        for k in (2, 1, 0):
            v = fma(v, F32(2.0 ** -8), Lf[k])
        T = Q(v) * Fraction(2) ** (e + f - 14)
        exact = sum(Q(a) * Q(b) for a, b in zip(x, c))
        scale = Fraction(2) ** e * max(abs(Q(cv)) for cv in c)
        bound = sum(abs(Q(a) * Q(b)) for a, b in zip(x, c)) / 2 ** 23 + scale / 2 ** 26
        err = abs(T - exact)
        worst = max(worst, float(err / scale))
        assert err <= bound
    # four products per term at the largest digits, 32 terms of a p2 box
    assert 32 * 4 * 256 * 128 < 2 ** 24
    print(f"worst |T - sum x c| / (2^e max|c|) = 2^{np.log2(worst):.1f}")
