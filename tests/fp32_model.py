"""Exact FP32 arithmetic on the host, for the CPU models of the kernels'
FP32 steps: values as numpy float32, every operation evaluated exactly in
rational arithmetic and rounded once to the nearest FP32 value (ties to
even), as IEEE FP32 add, multiply and fused multiply-add do."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def Q(x):
    """The exact rational value of an FP32 or FP64 number."""
    return Fraction(float(x))


def f32(q):
    """The FP32 value nearest to the rational q (ties to even), for the
    magnitudes the models use (no overflow, no subnormals)."""
    q = Fraction(q)
    if q == 0:
        return F32(0.0)
    s = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    scaled = q / Fraction(2) ** (e - 23)        # in [2^23, 2^24)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return F32(s * float(Fraction(m) * Fraction(2) ** (e - 23)))


def fma(a, b, c):
    """fmaf: a b + c rounded once."""
    return f32(Q(a) * Q(b) + Q(c))


def add(a, b):
    return f32(Q(a) + Q(b))


def sub(a, b):
    return f32(Q(a) - Q(b))


def mul(a, b):
    return f32(Q(a) * Q(b))
