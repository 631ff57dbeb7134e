// Double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers, normalised so
// that hi = fl32(hi + lo); it carries about 48 significant bits.  On this part
// an FP32 instruction issues at 64 times the FP64 rate, so a double-float
// operation of 3-12 FP32 instructions is still several times cheaper than one
// FP64 instruction.
//
// The building blocks are the classical error-free transformations: Knuth's
// TwoSum (a + b = s + e exactly), Dekker's Fast2Sum (the same when |a| >= |b|)
// and the FMA-based TwoProduct (a * b = p + e exactly).  The compound
// operations are the plain double-word algorithms ("sloppy" addition,
// double-word times double-word) as analysed by Joldes, Muller and Popescu
// (ACM TOMS 2017): each result is within a small multiple of 2^-48 of the
// operands' magnitudes, which is what residuals of least-squares systems need.
// Every step uses an explicit round-to-nearest intrinsic so that neither FMA
// contraction nor reassociation can alter the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace mvgd {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.0f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    const df p = two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    const df p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// acc + a * b
__device__ __forceinline__ df df_fma(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }

// a / b: one FP32 quotient, its remainder in double-float, one correction.
__device__ __forceinline__ df df_div(df a, df b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

// sqrt(a) for a >= 0: the FP32 root corrected by one Newton step on the
// double-float remainder a - s^2.
__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.0f)) return {__fsqrt_rn(fmaxf(a.hi, 0.0f)), 0.0f};
    const float s = __fsqrt_rn(a.hi);
    const df e = df_sub(a, two_prod(s, s));
    return fast_two_sum(s, __fdiv_rn(e.hi, __fmul_rn(2.0f, s)));
}

__device__ __forceinline__ bool df_less(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_from_double(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ bool df_isfinite(df a) { return isfinite(a.hi) && isfinite(a.lo); }

}  // namespace mvgd
