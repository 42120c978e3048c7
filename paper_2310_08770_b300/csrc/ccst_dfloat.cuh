// ccst_dfloat.cuh -- double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits. The building blocks are the classic error-free
// transformations: Knuth's TwoSum (the rounding error of a + b, exactly, in six
// additions), Dekker's FastTwoSum (the same when |a| >= |b|, three additions) and
// the FMA form of TwoProd (the error of a * b is fma(a, b, -a*b)). The add and
// multiply below are the standard double-word algorithms built from them
// (accurate sum, then renormalisation; product with the two cross terms folded
// into the error). On this GPU FP64 issues at a small fraction of the FP32 rate,
// so precision beyond FP32 is cheaper here than in native double.
#pragma once

#include <cuda_runtime.h>

namespace ccst {

struct df { float hi, lo; };
struct dfc { df re, im; };          // complex double-float

__device__ __forceinline__ df df_make(float x) { return {x, 0.f}; }

__device__ __forceinline__ df df_from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker FastTwoSum, |a| >= |b|.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_add(df a, df b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return {s, e};
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// The cheaper double-word sum (one TwoSum on the high parts, the low parts added in FP32,
// one renormalisation): its error is bounded absolutely, by about 2^-46 (|a| + |b|), not
// relative to |a + b|. That is the bound an FFT or a long dot product needs (errors measured
// against the magnitudes being combined), at about half the cost of df_add.
__device__ __forceinline__ df df_add_abs(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    fast_two_sum(s, e, s, e);
    return {s, e};
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s;
    fast_two_sum(p, e, s, e);
    return {s, e};
}
__device__ __forceinline__ df df_scale(df a, float k) {   // k a power of two: exact
    return {a.hi * k, a.lo * k};
}

// complex double-word arithmetic with the absolute-error sum (FFT butterflies, phases)
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return {df_add_abs(a.re, b.re), df_add_abs(a.im, b.im)}; }
__device__ __forceinline__ dfc csub(dfc a, dfc b) {
    return {df_add_abs(a.re, df_neg(b.re)), df_add_abs(a.im, df_neg(b.im))};
}
__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
    return {df_add_abs(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add_abs(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dfc cconj(dfc a) { return {a.re, df_neg(a.im)}; }

}  // namespace ccst
