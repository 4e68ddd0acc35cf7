"""The mixed forms' energy epilogue on FP32 pairs, modelled on the host with
every FP32 rounding reproduced: the accuracy its kernels and GPU tolerances
rest on, checked without a GPU.

The arithmetic, as the second-half kernels perform it per occupied pair
(i, j) and lane a, over the virtual orbitals b (Sec. II.C energy tensor,
Eq. (ed2) with T = v D):

* e_i + e_j - e_a in FP64, split into an FP32 pair (h, l), and e_b likewise;
* x = (e_i + e_j - e_a) - e_b as a pair (TwoSum of the high parts);
* D = 1/x: an FP32 reciprocal estimate, one FP32 Newton step, then one step
  on the pair;
* E_J term v^2 D and E_K term v vk D, v^2 and v vk rounded to FP32, each
  product with D split exactly (Dekker's TwoProduct by an FMA) and added to a
  pair accumulator by TwoSum, renormalised after every term;
* even and odd b in separate accumulators, each flushed to FP64 once per pair.

Checked here: D to 2^-44 relative; the pair sums of the 27 terms of a lane
to 2^-43 of their size against exact rational arithmetic; and that dropping
the low part of D, or TwoProduct's error term, breaks those bounds.  Also the
FP64E second half's pair multiply-add: 32-term dot products of FP64 values
carried as pairs within 2^-43 of sum |a b|.
"""
from fractions import Fraction

import numpy as np

from fp32_model import F32, Q, add, f32, fma, mul, sub


def two_sum(a, b):
    s = add(a, b)
    bp = sub(s, a)
    return s, add(sub(a, sub(s, bp)), sub(b, bp))


def split(x):
    """An FP64 value as an FP32 pair: h, then the FP32 rounding of x - h."""
    h = f32(Q(x))
    return (h, f32(Q(np.float64(x) - np.float64(h))))


def pair_sub(a, b):
    s, e = two_sum(a[0], -b[0])
    e = add(e, sub(a[1], b[1]))
    h = add(s, e)
    return (h, sub(e, sub(h, s)))


def pair_rcp(x, keep_low=True):
    r = f32(1 / Q(x[0]))                         # the reciprocal estimate, modelled as rounded
    r = fma(r, fma(-x[0], r, F32(1.0)), r)
    e = fma(-x[0], r, F32(1.0))
    if keep_low:
        e = fma(-x[1], r, e)
    return (r, mul(r, e))


def pair_acc(s, w, D, exact_product=True):
    ph = mul(w, D[0])
    pl = fma(w, D[1], fma(w, D[0], -ph)) if exact_product else mul(w, D[1])
    t, e = two_sum(s[0], ph)
    e = add(e, add(s[1], pl))
    h = add(t, e)
    return (h, sub(e, sub(h, t)))


def lane_sums(eija, eb, v, vk, keep_low=True, exact_product=True):
    """One lane's E_J and E_K sums over b, even and odd b apart, in FP64."""
    xs = split(eija)
    acc = {k: [(F32(0), F32(0)), (F32(0), F32(0))] for k in "JK"}
    Ds = []
    for b in range(len(eb)):
        D = pair_rcp(pair_sub(xs, split(eb[b])), keep_low)
        Ds.append(D)
        p = b % 2
        acc["J"][p] = pair_acc(acc["J"][p], mul(v[b], v[b]), D, exact_product)
        acc["K"][p] = pair_acc(acc["K"][p], mul(v[b], vk[b]), D, exact_product)
    out = {}
    for k in "JK":
        out[k] = sum((float(np.float64(h) + np.float64(l)) for h, l in acc[k]), 0.0)
    return out, Ds


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        eocc = -rng.uniform(0.3, 1.5, 2)                 # e_i, e_j
        ea = rng.uniform(0.05, 3.0)
        eb = rng.uniform(0.05, 3.0, 27)
        eija = (eocc[0] + eocc[1]) - ea                   # FP64, as in the kernels
        v = (rng.standard_normal(27) * 10.0 ** rng.uniform(-5, -2, 27)).astype(F32)
        vk = (rng.standard_normal(27) * 10.0 ** rng.uniform(-6, -3, 27)).astype(F32)
        yield eija, eb, v, vk


def _errors(keep_low=True, exact_product=True, n=40):
    worst_D, worst_J, worst_K = 0.0, 0.0, 0.0
    for eija, eb, v, vk in _cases(n, seed=11):
        got, Ds = lane_sums(eija, eb, v, vk, keep_low, exact_product)
        ex_J = Fraction(0)
        ex_K = Fraction(0)
        absK = Fraction(0)
        for b in range(len(eb)):
            # the exact denominator of the FP64 inputs as the kernel reads them
            Dx = 1 / (Q(eija) - Q(eb[b]))
            worst_D = max(worst_D, float(abs(Q(Ds[b][0]) + Q(Ds[b][1]) - Dx) / abs(Dx)))
            ex_J += Q(mul(v[b], v[b])) * Dx
            ex_K += Q(mul(v[b], vk[b])) * Dx
            absK += abs(Q(mul(v[b], vk[b])) * Dx)
        worst_J = max(worst_J, float(abs(Q(got["J"]) - ex_J) / abs(ex_J)))
        worst_K = max(worst_K, float(abs(Q(got["K"]) - ex_K) / absK))
    return worst_D, worst_J, worst_K


def test_pair_epilogue_reaches_its_bounds():
    d, j, k = _errors()
    print(f"D 2^{np.log2(d):.1f}, E_J sum 2^{np.log2(j):.1f}, E_K sum 2^{np.log2(k):.1f} (relative)")
    assert d <= 2.0 ** -44
    assert j <= 2.0 ** -43
    assert k <= 2.0 ** -43            # relative to the sum of the terms' magnitudes (E_K terms change sign)


def test_each_pair_step_is_needed():
    # without the low part of x in the reciprocal, D keeps only FP32 accuracy
    d, j, _ = _errors(keep_low=False, n=10)
    assert d > 2.0 ** -30 and j > 2.0 ** -30
    # without TwoProduct's error term, each product keeps only FP32 accuracy
    _, j, _ = _errors(exact_product=False, n=10)
    assert j > 2.0 ** -30


def pair_mac(s, a, b):
    """s += a b for pairs a, b: TwoProduct of the high parts, the cross terms
    in the low part (a.l b.l dropped), TwoSum into s, renormalised -- the
    FP64E second half's multiply-add."""
    ph = mul(a[0], b[0])
    pl = fma(a[1], b[0], fma(a[0], b[1], fma(a[0], b[0], -ph)))
    t, e = two_sum(s[0], ph)
    e = add(e, add(s[1], pl))
    h = add(t, e)
    return (h, sub(e, sub(h, t)))


def test_pair_dot_products_of_the_fp64e_second_half():
    """32-term dot products of FP64 values carried as pairs (the FP64E virtual
    quarter transformations) within 2^-43 of sum |a b|; without the cross
    terms they fall to FP32 accuracy."""
    rng = np.random.default_rng(12)
    worst, worst_nocross = 0.0, 0.0
    for _ in range(30):
        a = rng.standard_normal(32) * 10.0 ** rng.uniform(-4, 0, 32)
        b = rng.standard_normal(32) * 10.0 ** rng.uniform(-2, 0, 32)
        ap = [split(v) for v in a]
        bp = [split(v) for v in b]
        s = (F32(0), F32(0))
        s2 = (F32(0), F32(0))
        for x, y in zip(ap, bp):
            s = pair_mac(s, x, y)
            s2 = pair_mac(s2, (x[0], F32(0)), (y[0], F32(0)))
        exact = sum(Q(x) * Q(y) for x, y in zip(a, b))
        mag = sum(abs(Q(x) * Q(y)) for x, y in zip(a, b))
        worst = max(worst, float(abs(Q(s[0]) + Q(s[1]) - exact) / mag))
        worst_nocross = max(worst_nocross, float(abs(Q(s2[0]) + Q(s2[1]) - exact) / mag))
    print(f"pair dot products: 2^{np.log2(worst):.1f} of sum|ab| (high parts only: 2^{np.log2(worst_nocross):.1f})")
    assert worst <= 2.0 ** -43
    assert worst_nocross > 2.0 ** -30
