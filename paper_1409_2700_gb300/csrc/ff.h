// ff.h -- FP32 pairs: 48-bit double-length arithmetic on the FP32 pipes.
#pragma once
#include "convert.h"

namespace mcpt {

// FP32 pairs: an unevaluated sum h + l of two FP32 values with |l| <= ulp(h)
// (Dekker's double-length arithmetic, Numer. Math. 18 (1971) 224) carries 48
// significant bits on the FP32 pipes, which GB300 runs at 64x its FP64 rate.
// The mixed forms' energy epilogue and the FP64-emulating tensor-core form
// use them; every rounding is named (explicit _rn operations, so that the
// compiler contracts none of them into an FMA, which would break the
// error-free steps).
struct __align__(8) FF {
    float h, l;
};

// x (an FP64 value of FP32 range) as a pair: h rounded to FP32, l the FP32
// rounding of the remainder; |x - (h + l)| <= 2^-48 |x|.  One FP64 subtraction.
__device__ __forceinline__ FF ff_split(double x)
{
    const float h = f32_from_f64(x);
    return FF{h, f32_from_f64(x - f64_from_f32(h))};
}

// s + e = a + b exactly (Knuth's TwoSum, no condition on |a|, |b|)
__device__ __forceinline__ float two_sum(float a, float b, float& e)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return s;
}

// a - b for pairs whose difference does not cancel (a <= 0 <= b, which holds
// for e_i + e_j - e_a and e_b of any system with a positive gap): absolute
// error below 2^-47 (|a| + |b|), so relative error below 2^-46 here.
__device__ __forceinline__ FF ff_sub(FF a, FF b)
{
    float e;
    const float s = two_sum(a.h, -b.h, e);
    e = __fadd_rn(e, __fsub_rn(a.l, b.l));
    const float h = __fadd_rn(s, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

// 1/x for a pair x: the FP32 reciprocal estimate r, one FP32 Newton step
// (|1 - x r| <~ 2^-23), then 1/x = r / (1 - eps) ~= r + r eps with
// eps = 1 - x r evaluated to the pair's precision: relative error ~2^-45.
__device__ __forceinline__ FF ff_rcp(FF x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.h));
    r = fmaf(r, fmaf(-x.h, r, 1.f), r);
    float e = fmaf(-x.h, r, 1.f);
    e = fmaf(-x.l, r, e);
    return FF{r, __fmul_rn(r, e)};
}

// s += w D, w an FP32 value: the product w D.h split exactly by an FMA
// (Dekker's TwoProduct), w D.l added to its low part, then TwoSum into the
// accumulator and a renormalisation, so |s.l| <= ulp(s.h) after every term.
__device__ __forceinline__ void ff_acc(FF& s, float w, FF D)
{
    const float ph = __fmul_rn(w, D.h);
    const float pl = fmaf(w, D.l, fmaf(w, D.h, -ph));
    float e;
    const float t = two_sum(s.h, ph, e);
    e = __fadd_rn(e, __fadd_rn(s.l, pl));
    s.h = __fadd_rn(t, e);
    s.l = __fsub_rn(e, __fsub_rn(s.h, t));
}

__device__ __forceinline__ double ff_f64(FF s) { return f64_from_f32(s.h) + f64_from_f32(s.l); }

// s += a b for pairs a and b: the product a.h b.h split exactly by an FMA, the
// cross terms a.h b.l + a.l b.h added to its low part (a.l b.l, below 2^-48 of
// the product, is dropped), then TwoSum into the accumulator and a
// renormalisation, as in ff_acc.
__device__ __forceinline__ void ff_mac(FF& s, FF a, FF b)
{
    const float ph = __fmul_rn(a.h, b.h);
    const float pl = fmaf(a.l, b.h, fmaf(a.h, b.l, fmaf(a.h, b.h, -ph)));
    float e;
    const float t = two_sum(s.h, ph, e);
    e = __fadd_rn(e, __fadd_rn(s.l, pl));
    s.h = __fadd_rn(t, e);
    s.l = __fsub_rn(e, __fsub_rn(s.h, t));
}

// a b for pairs, renormalised (TwoProduct of the high parts, cross terms in
// the low part; a.l b.l dropped).
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const float ph = __fmul_rn(a.h, b.h);
    const float pl = fmaf(a.l, b.h, fmaf(a.h, b.l, fmaf(a.h, b.h, -ph)));
    const float h = __fadd_rn(ph, pl);
    return FF{h, __fsub_rn(pl, __fsub_rn(h, ph))};
}

// s renormalised: |l| <= ulp(h) / 2, the same value to FP32 rounding of l.
__device__ __forceinline__ FF ff_norm(FF s)
{
    const float h = __fadd_rn(s.h, s.l);
    return FF{h, __fsub_rn(s.l, __fsub_rn(h, s.h))};
}

// ff_mac without the renormalisation: s.l gathers the TwoSum errors and the
// products' low parts; renormalise (ff_norm) every few terms -- after k terms
// |s.l| is below k ulp(s.h), so its own roundings stay below k^2 2^-49 |s|.
__device__ __forceinline__ void ff_mac_nr(FF& s, FF a, FF b)
{
    const float ph = __fmul_rn(a.h, b.h);
    const float pl = fmaf(a.l, b.h, fmaf(a.h, b.l, fmaf(a.h, b.h, -ph)));
    float e;
    s.h = two_sum(s.h, ph, e);
    s.l = __fadd_rn(s.l, __fadd_rn(e, pl));
}

// a + b for pairs: TwoSum of the high parts, the low parts added, renormalised.
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    float e;
    const float t = two_sum(a.h, b.h, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(t, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, t))};
}

}  // namespace mcpt
