// convert.h -- FP64 -> FP32/TF32 conversions on the integer pipes.
//
// On GB300 the FP64 unit is a small fraction of the FP32 one, and a
// cvt.f32.f64 issues on it; streaming every AO integral through that unit
// caps the transform far below the memory roofline.  These helpers build the
// IEEE-754 result from the binary64 bit fields with integer operations
// instead (sign | exponent rebiased by 1023-127 = 896 | leading mantissa
// bits, rounded half away from zero on the first dropped bit).  Magnitudes
// below 2^-126 flush to (signed) zero; inputs are assumed finite and below
// 2^127, which the integrals and coefficients are.
#pragma once
#include <cuda_runtime.h>

namespace mcpt {

// TF32 (returned as FP32 bits with the 13 low mantissa bits zero) from the
// high 32 bits of a double: TF32 keeps 10 mantissa bits, and rounding half
// away from zero only needs the first dropped bit, which lies in the high word.
__device__ __forceinline__ unsigned tf32_from_f64_hi(unsigned hi)
{
    const unsigned sign = hi & 0x80000000u;
    const unsigned r = ((hi & 0x7FFFFFFFu) + (1u << 9)) >> 10;   // exponent(11) | mantissa(10), rounded
    const int e = (int)(r >> 10) - 896;
    return e > 0 ? (sign | ((r - (896u << 10)) << 13)) : sign;
}

// FP32 from both words of a double, round half away from zero.
__device__ __forceinline__ float f32_from_f64_bits(unsigned lo, unsigned hi)
{
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;
    unsigned m = ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    m += (lo >> 28) & 1u;
    return __uint_as_float(e > 0 ? (sign | m) : sign);
}

__device__ __forceinline__ float f32_from_f64(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return f32_from_f64_bits((unsigned)b, (unsigned)(b >> 32));
}

// FP64 from FP32 bits (exact), integer pipes only; zero and FP32 denormals -> zero.
__device__ __forceinline__ double f64_from_f32(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned hi = e ? (sign | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)) : sign;
    const unsigned lo = (u & 7u) << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// FP32 reciprocal seed of an FP64 value, widened back to FP64: conversions on
// the integer pipes, rcp.approx.ftz.f32 on the special-function unit.  For |x|
// in a normal FP32 range its relative error is below 2^-22 (rounding x to
// FP32 plus the approximate reciprocal).
__device__ __forceinline__ double rcp_seed_f64(double x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f32_from_f64(x)));
    return f64_from_f32(r);
}

// v / x in FP64 by Newton-Raphson on the reciprocal, r <- r + r(1 - x r),
// from the FP32 seed; each step squares the relative error.  The last step is
// folded into the product: with e = 1 - x r, v/x ~= (v r) + (v r) e, so STEPS
// steps cost 2 STEPS + 1 FP64 operations.  One step leaves ~2^-44 (6e-14),
// two reach FP64 rounding.
template <int STEPS>
__device__ __forceinline__ double div_newton(double v, double x)
{
    double r = rcp_seed_f64(x);
#pragma unroll
    for (int k = 0; k + 1 < STEPS; k++) r = fma(r, fma(-x, r, 1.0), r);
    const double e = fma(-x, r, 1.0);
    const double t = v * r;
    return fma(t, e, t);
}

}  // namespace mcpt
