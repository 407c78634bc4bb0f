// Double-FP32 ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers, a significand of about 48 bits with FP32's
// exponent range.  GB300 issues FP32 FMAs at 64x its FP64 rate, so a
// multiply-accumulate of ~12 FP32 operations still runs several times
// faster than one FP64 FMA.
//
// The product uses the exact FMA residual of the leading parts
// (p = fl(a.hi b.hi), e = a.hi b.hi - p exactly) and the two cross terms;
// the sum is Knuth's branch-free two-sum (exact for any operand order).  The
// accumulator is left unnormalised (hi, lo with |lo| of the order of a few
// ulp(hi) after many steps), which keeps each multiply-accumulate at 12
// operations; df_norm renormalises.  The __f*_rn intrinsics keep the
// compiler from contracting the error-free transformations into FMAs.
#pragma once

#include <cstdint>

struct __align__(8) df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float v) : hi(v), lo(0.f) {}
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
};

__host__ __device__ __forceinline__ df df_from(double v) {
    const float h = (float)v;
    return df(h, (float)(v - (double)h));
}
__host__ __device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

// a * b + c
__device__ __forceinline__ df fma(df a, df b, df c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // exact: a.hi b.hi = p + e
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(c.hi, p);    // two-sum: c.hi + p = s + err exactly
    const float bb = __fsub_rn(s, c.hi);
    const float err = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    return df(s, __fadd_rn(c.lo, __fadd_rn(e, err)));
}

__device__ __forceinline__ df df_norm(df a) {
    const float s = __fadd_rn(a.hi, a.lo);
    return df(s, __fsub_rn(a.lo, __fsub_rn(s, a.hi)));
}
