"""The digit scheme of the FP64-emulating tensor-core form (MCPT_FP64E),
modelled on the host in exact rational arithmetic: the claims its kernel and
its GPU tolerances rest on, checked without a GPU.

The scheme, as the kernel implements it:

* An FP64 vector (32 integrals of one row chunk, or a C_Y column) is held in
  48-bit fixed point relative to its largest exponent field e_max:
  N = floor(|x| 2^(47 - e)), e = e_max - 1023, as six unsigned bytes
  N = sum_u d_u 2^(40 - 8u), each carrying the element's sign.
* The tensor cores sum the digit products by level, L_k = sum_{u+v=k} sum_p
  d_u(x_p) d_v(c_p), in FP32.  That sum is exact only while |L_k| < 2^24.
* The levels kept are 0-6; T = 2^(e_x + e_c - 14) sum_k L_k 2^(-8k).

Checked here:

1. every level sum stays below 2^24 (exact tensor-core sums);
2. levels 0-6 leave |T - sum x c| within 2^-44 max|x| max|c| (the bound the
   GPU tests' 1e-12 per dimer rests on), and dropping level 6 would not;
3. the fixed point alone (all levels) is within the truncation bound.
"""
import math
import struct
from fractions import Fraction

import numpy as np


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _exp_field(x):
    return (_bits(x) >> 52) & 0x7FF


def _fx48(x, emax):
    """floor(|x| 2^(47 - e)) from the bit fields, as the kernel does."""
    b = _bits(x)
    ex = (b >> 52) & 0x7FF
    if ex == 0:
        return 0
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    s = emax - ex + 5
    return m >> s if s < 64 else 0


def _digits(x, emax):
    N = _fx48(x, emax)
    sg = -1 if x < 0 else 1
    return [sg * ((N >> (40 - 8 * u)) & 255) for u in range(6)]


def _chunks(n_chunks, seed):
    rng = np.random.default_rng(seed)
    for t in range(n_chunks):
        x = rng.standard_normal(32) * 10.0 ** rng.uniform(-6, 2, 32)
        c = rng.standard_normal(32) * 10.0 ** rng.uniform(-3, 0, 32)
        if t % 5 == 0:
            x[rng.integers(0, 32, 6)] = 0.0
        yield x, c


def _levels(dx, dc, kmax):
    return [sum(dx[p][u] * dc[p][k - u] for p in range(len(dx)) for u in range(max(0, k - 5), min(k, 5) + 1))
            for k in range(kmax)]


def test_level_sums_are_exact_in_fp32():
    """Every digit-product level sum of a 32-element chunk stays below 2^24
    (seven levels, at most 7 x 32 products of magnitude below 2^16 each)."""
    worst = 0
    for x, c in _chunks(150, seed=3):
        ex = max(_exp_field(v) for v in np.abs(x))
        ec = max(_exp_field(v) for v in np.abs(c))
        L = _levels([_digits(v, ex) for v in x], [_digits(v, ec) for v in c], 7)
        worst = max(worst, max(abs(l) for l in L))
    assert worst < 2 ** 24
    # the bound holds for any digits: (k + 1) * 32 * 255^2 < 2^24 up to k = 6
    assert 7 * 32 * 255 * 255 < 2 ** 24


def test_levels_zero_to_six_reach_the_fp64_bound():
    worst7, worst6, worst_fx = 0.0, 0.0, 0.0
    for x, c in _chunks(150, seed=5):
        ex = max(_exp_field(v) for v in np.abs(x))
        ec = max(_exp_field(v) for v in np.abs(c))
        e, f = ex - 1023, ec - 1023
        dx = [_digits(v, ex) for v in x]
        dc = [_digits(v, ec) for v in c]
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, c))
        scale = float(np.max(np.abs(x)) * np.max(np.abs(c)))

        def T(kmax):
            L = _levels(dx, dc, kmax)
            return Fraction(2) ** (e + f - 14) * sum(Fraction(L[k]) / Fraction(256) ** k for k in range(kmax))

        Nx = [(-1 if v < 0 else 1) * _fx48(v, ex) for v in x]
        Nc = [(-1 if v < 0 else 1) * _fx48(v, ec) for v in c]
        fixed = Fraction(2) ** (e + f - 94) * sum(a * b for a, b in zip(Nx, Nc))
        worst7 = max(worst7, abs(float(T(7) - exact)) / scale)
        worst6 = max(worst6, abs(float(T(6) - exact)) / scale)
        worst_fx = max(worst_fx, abs(float(fixed - exact)) / scale)
    print(f"levels 0-6: 2^{math.log2(worst7):.1f}, levels 0-5: 2^{math.log2(worst6):.1f}, "
          f"fixed point alone: 2^{math.log2(worst_fx):.1f} of max|x| max|c|")
    # truncation of each element to 2^-47 of its vector's power of two, both
    # operands, 32 terms: at most 2 * 32 * 2^-47 * 2 = 2^-40 (typically far less)
    assert worst_fx <= 2.0 ** -40
    assert worst7 <= 2.0 ** -44
    # level 6 is needed: without it the error is several times larger
    assert worst6 > 4 * worst7


def test_level_combination_on_pairs():
    """The epilogue's combination of the seven level sums into an FP32 pair,
    modelled with every FP32 rounding: levels 6-4 by two FP32 FMAs, level 3
    by a third, levels 2-0 by exact scalings and TwoSums with the errors
    gathered in the low word, one renormalisation at the end.  The FP32
    rounding of levels 6-3 carries weight 2^-24, so the error is absolute in
    level-0 units: within 2^-23 of the exact sum_k L_k 2^(-8k), i.e. 2^-47 of
    the fixed point's full scale 2^24 -- the size of the digits' own
    truncation, whatever cancellation leaves of the sum."""
    from fp32_model import F32, Q as q32, add, fma, mul, sub

    def two_sum(a, b):
        s = add(a, b)
        bp = sub(s, a)
        return s, add(sub(a, sub(s, bp)), sub(b, bp))

    rng = np.random.default_rng(13)
    worst = 0.0
    lim = 7 * 32 * 255 * 255
    for t in range(400):
        L = [F32(float(v)) for v in rng.integers(-lim, lim + 1, 7)]
        if t % 3 == 0:
            L[0] = F32(0.0)                          # a cancelled top level
        h = fma(fma(L[6], F32(2.0 ** -8), L[5]), F32(2.0 ** -8), L[4])
        h = fma(h, F32(2.0 ** -8), L[3])
        lo = F32(0.0)
        for k in (2, 1, 0):
            h, e = two_sum(L[k], mul(h, F32(2.0 ** -8)))
            lo = fma(lo, F32(2.0 ** -8), e)
        hn = add(h, lo)
        ln = sub(lo, sub(hn, h))
        exact = sum(q32(L[k]) / Fraction(256) ** k for k in range(7))
        worst = max(worst, float(abs(q32(hn) + q32(ln) - exact)))
    print(f"level combination: 2^{math.log2(worst):.1f} level-0 units")
    assert worst <= 2.0 ** -23
