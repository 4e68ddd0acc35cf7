"""The compensated-FP32 form's first half (MCPT_FP32C), modelled on the host
with every FP32 rounding reproduced and checked against exact rational
arithmetic without a GPU.

Per output (row (p1, p3), occupied pair (i, j)) the kernel forms
  H = sum_{p0} C_X[p0][i] F(p0),  F(p0) = sum_{p2} C_Y[p2][j] E[p0][p1][p2][p3],
with the integrals rounded once to FP32 and both sums accumulated by Dot2
(Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
Comput. 26, 2005): each product split exactly by an FMA (TwoProduct), each
addition's error kept by TwoSum, the errors gathered in a low word; the
inner sum stays an unevaluated pair (hi, lo) and enters the outer sum as
w hi (TwoProduct) plus w lo (one FMA); the result is hi + lo rounded once.

Dot2's bound for such a sum is one rounding of the result plus a term
quadratic in the unit roundoff: |H - exact| <= 2^-24 |exact| + c n^2 2^-48
sum |w u e|.  Checked here with c n^2 = 2^8 (n = 32 terms per level); and a
plain FP32 accumulation of the same sums is shown to miss that bound.
"""
from fractions import Fraction

import numpy as np

from fp32_model import F32, Q, add, f32, fma, mul, sub


def two_sum(a, b):
    s = add(a, b)
    z = sub(s, a)
    return s, add(sub(a, sub(s, z)), sub(b, z))


def dot2_step(acc, x, y):
    h = mul(x, y)
    r = fma(x, y, -h)
    s, q = two_sum(acc[0], h)
    return (s, add(acc[1], add(q, r)))


def dot2_step_pair(acc, w, v):
    acc = dot2_step(acc, w, v[0])
    return (acc[0], fma(w, v[1], acc[1]))


def plain_step(acc, x, y):
    return (fma(x, y, acc[0]), acc[1])


def h_value(CX, CY, E, step=dot2_step):
    """One output: CX[p0] (FP32), CY[p2] (FP32), E[p0][p2] (FP32)."""
    acc = (F32(0), F32(0))
    for p0 in range(E.shape[0]):
        F = (F32(0), F32(0))
        for p2 in range(E.shape[1]):
            F = step(F, CY[p2], E[p0, p2])
        acc = dot2_step_pair(acc, CX[p0], F) if step is dot2_step else plain_step(acc, CX[p0], add(F[0], F[1]))
    return add(acc[0], acc[1])


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        E = (rng.standard_normal((32, 32)) * 10.0 ** rng.uniform(-6, 0, (32, 32))).astype(np.float64)
        E = np.array([[f32(Q(v)) for v in row] for row in E], dtype=np.float32)   # rounded once to FP32
        CX = rng.standard_normal(32).astype(np.float32)
        CY = rng.standard_normal(32).astype(np.float32)
        yield CX, CY, E


def _check(step):
    worst = 0.0
    ok = True
    for CX, CY, E in _cases(25, seed=9):
        exact = sum(Q(CX[p0]) * Q(CY[p2]) * Q(E[p0, p2]) for p0 in range(32) for p2 in range(32))
        mag = sum(abs(Q(CX[p0]) * Q(CY[p2]) * Q(E[p0, p2])) for p0 in range(32) for p2 in range(32))
        err = abs(Q(h_value(CX, CY, E, step)) - exact)
        bound = abs(exact) / 2 ** 24 + mag / 2 ** 40
        worst = max(worst, float(err / mag))
        ok = ok and err <= bound
    return ok, worst


def test_dot2_reaches_its_bound():
    ok, worst = _check(dot2_step)
    print(f"Dot2: worst |H - exact| / sum|w u e| = 2^{np.log2(worst):.1f}")
    assert ok


def test_plain_fp32_accumulation_misses_it():
    ok, _ = _check(plain_step)
    assert not ok
