// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, about 48 significant bits, computed on the
// FP32 pipe.  Error-free transformations after Knuth (TwoSum), Dekker
// (FastTwoSum) and the fused multiply-add product (TwoProd).
#pragma once

#include <cuda_runtime.h>

namespace ftcj {

struct df {
    float hi, lo;
};

struct cdf {  // complex double-float
    df re, im;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

__host__ __device__ inline df df_from_double(double x) {
    float hi = (float)x;
    float lo = (float)(x - (double)hi);
    return df{hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// |a| >= |b| or a == 0
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// double-float times an FP32 value
__device__ __forceinline__ df df_mulf(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

// a*b - c*d and a*b + c*d with one renormalisation each
__device__ __forceinline__ df df_mul_sub(df a, df b, df c, df d) {
    float p1 = __fmul_rn(a.hi, b.hi);
    float e1 = __fmaf_rn(a.hi, b.hi, -p1);
    float p2 = __fmul_rn(c.hi, d.hi);
    float e2 = __fmaf_rn(c.hi, d.hi, -p2);
    df s = two_sum(p1, -p2);
    float e = __fadd_rn(s.lo, __fsub_rn(e1, e2));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(-c.hi, d.lo, e);
    e = __fmaf_rn(-c.lo, d.hi, e);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_mul_add(df a, df b, df c, df d) {
    float p1 = __fmul_rn(a.hi, b.hi);
    float e1 = __fmaf_rn(a.hi, b.hi, -p1);
    float p2 = __fmul_rn(c.hi, d.hi);
    float e2 = __fmaf_rn(c.hi, d.hi, -p2);
    df s = two_sum(p1, p2);
    float e = __fadd_rn(s.lo, __fadd_rn(e1, e2));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(c.hi, d.lo, e);
    e = __fmaf_rn(c.lo, d.hi, e);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    return cdf{df_mul_sub(a.re, b.re, a.im, b.im), df_mul_add(a.re, b.im, a.im, b.re)};
}

// complex times real double-float
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return cdf{df_mul(a.re, s), df_mul(a.im, s)}; }

__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }

__device__ __forceinline__ cdf cdf_conj(cdf a) { return cdf{a.re, df_neg(a.im)}; }

}  // namespace ftcj
