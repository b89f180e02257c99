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

// x = hi + lo to 48 bits.  Done on the integer pipe: hi keeps the sign, the exponent and the top 23
// mantissa bits of x (truncation), lo is the value of the 29 bits cut off; only |x| outside the FP32
// normal range takes the FP64 route (FP64 conversions and subtraction run on the FP64 pipe, which on
// this GPU is ~1/64 of the FP32 rate and would otherwise dominate the staging of pair amplitudes).
__device__ __forceinline__ F2 f2_split(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int h = (unsigned int)(b >> 32), l = (unsigned int)b;
    const int e = (int)((h >> 20) & 0x7FFu);  // biased FP64 exponent
    if (e < 1023 - 126 || e > 1023 + 127) {
        const float hi = __double2float_rn(x);
        return F2(hi, __double2float_rn(x - (double)hi));
    }
    const unsigned int sign = h & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
    const float lo = ldexpf(__uint2float_rn(l & 0x1FFFFFFFu), e - 1023 - 52);
    return F2(hi, sign ? -lo : lo);
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
