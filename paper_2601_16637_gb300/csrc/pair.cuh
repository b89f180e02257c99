#pragma once
// FP64-accurate arithmetic on the FP32 pipe: a value is the unevaluated sum hi + lo of two floats.
// Products are exact hi*hi (a fused multiply-add recovers its rounding error, Dekker's product) plus
// the two cross terms; sums use Knuth's two-sum.  On GB300 the FP32 pipe is ~64x the FP64 pipe, so
// the FP64-accurate sigma and the Davidson solver's Ritz combinations run on these pairs.

#include "common.cuh"

namespace sbd {

// A value hi + lo of two floats (|lo| <= ulp(hi)/2 after renormalisation).
struct F2 {
    float hi, lo;
    F2() = default;
    __host__ __device__ constexpr F2(float h) : hi(h), lo(0.f) {}
    __host__ __device__ constexpr F2(float h, float l) : hi(h), lo(l) {}
};

// x = hi + lo to 48 bits, on the integer and FP32 pipes only, without branches.  hi keeps the sign,
// the exponent and the top 23 mantissa bits of x (truncation); lo is the value of the 29 bits cut
// off, converted to FP32 and scaled by two exact power-of-two products.  Outside the FP32 normal
// range selects give: |x| < 2^-126 (zeros included) a signed zero, |x| >= 2^128 and infinities an
// infinity, NaN a NaN.  (An FP64 fallback or a branch here costs every element: the compiler
// if-converts the fallback, whose FP64 conversions run at ~1/64 of the FP32 rate on this GPU, and
// the streaming kernels of the solver spend most of their instructions in this split.)
__device__ __forceinline__ F2 f2_split(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int h = (unsigned int)(b >> 32), l = (unsigned int)b;
    const unsigned int sign = h & 0x80000000u, ha = h ^ sign;  // ha: high word of |x|
    const bool in = ha - 0x38100000u < 0x0FE00000u;             // biased FP64 exponent in [897, 1150]
    // in range, ha - (896 << 20) holds the FP32 exponent (1..254) above the top 20 mantissa bits
    const unsigned int t = (ha - 0x38000000u) << 3;
    const float lo = __uint2float_rn(l & 0x1FFFFFFFu) * 0x1p-52f * __uint_as_float(t & 0x7F800000u);
    const unsigned int big = sign | 0x7F800000u | ((ha | (unsigned int)(l != 0u)) > 0x7FF00000u ? 0x400000u : 0u);
    const unsigned int hb = in ? (sign | t | (l >> 29)) : (ha >= 0x47F00000u ? big : sign);
    const unsigned int lb = in ? (__float_as_uint(lo) ^ sign) : 0u;
    return F2(__uint_as_float(hb), __uint_as_float(lb));
}
__device__ __forceinline__ double f2_value(F2 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2(-a.hi, -a.lo); }

// acc += a * b.  The product's high part is exact to 48 bits (hi*hi and its rounding error from
// a fused multiply-add, plus the cross terms); it enters acc.hi through a two-sum whose error
// joins the low parts, which are gathered in acc.lo and renormalised by f2_add.  The explicit
// _rn intrinsics keep the compiler from fusing the two-sum into multiply-adds.
__device__ __forceinline__ void f2_mac(F2 &acc, F2 a, F2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// a + b: two-sum of the high parts, low parts added, renormalised
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    t = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, t);
    return F2(hi, __fsub_rn(t, __fsub_rn(hi, s)));
}

}  // namespace sbd
