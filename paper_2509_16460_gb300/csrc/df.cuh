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

// ---- deferred renormalisation --------------------------------------------
// The "_u" forms leave out the closing FastTwoSum: hi + lo is the same value
// to the same accuracy, but |lo| may exceed ulp(hi)/2 by a few units.  Every
// operation above accepts such operands (TwoSum of the high parts is exact for
// any inputs; the products carry a.lo b.hi and a.hi b.lo), so chains of a few
// steps in a hot loop renormalise once, with df_norm, before a value is kept.
__device__ __forceinline__ df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df df_add_u(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return df{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ df df_mulf_u(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df{p, e};
}

__device__ __forceinline__ df df_mul_u(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df{p, e};
}

__device__ __forceinline__ df df_mul_sub_u(df a, df b, df c, df d) {
    const float p1 = __fmul_rn(a.hi, b.hi);
    const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
    const float p2 = __fmul_rn(c.hi, d.hi);
    const float e2 = __fmaf_rn(c.hi, d.hi, -p2);
    const df s = two_sum(p1, -p2);
    float e = __fadd_rn(s.lo, __fsub_rn(e1, e2));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(-c.hi, d.lo, e);
    e = __fmaf_rn(-c.lo, d.hi, e);
    return df{s.hi, e};
}

__device__ __forceinline__ df df_mul_add_u(df a, df b, df c, df d) {
    const float p1 = __fmul_rn(a.hi, b.hi);
    const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
    const float p2 = __fmul_rn(c.hi, d.hi);
    const float e2 = __fmaf_rn(c.hi, d.hi, -p2);
    const df s = two_sum(p1, p2);
    float e = __fadd_rn(s.lo, __fadd_rn(e1, e2));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(c.hi, d.lo, e);
    e = __fmaf_rn(c.lo, d.hi, e);
    return df{s.hi, e};
}

__device__ __forceinline__ cdf cdf_mul_u(cdf a, cdf b) {
    return cdf{df_mul_sub_u(a.re, b.re, a.im, b.im), df_mul_add_u(a.re, b.im, a.im, b.re)};
}

__device__ __forceinline__ cdf cdf_add_u(cdf a, cdf b) { return cdf{df_add_u(a.re, b.re), df_add_u(a.im, b.im)}; }

__device__ __forceinline__ cdf cdf_scale_u(cdf a, df s) { return cdf{df_mul_u(a.re, s), df_mul_u(a.im, s)}; }

__device__ __forceinline__ cdf cdf_norm(cdf a) { return cdf{df_norm(a.re), df_norm(a.im)}; }

// ---- conversions that keep off the FP64 pipe ----------------------------
// GB300 issues FP64 (conversions included) at 2 lanes per clock per SM, so
// doubles are split into double-float and rebuilt from their exponent and
// mantissa fields with integer operations; only the final addition of
// join_df is an FP64 instruction.  Magnitudes below 2^-126 (the normal FP32
// range) are dropped on input and output: an absolute error below 2^-126.

// hi = x truncated to 24 significant bits, lo = the remaining 29 bits rounded
// to 24 (a subnormal FP32 number when x is below about 2^-74)
__device__ __forceinline__ df split_double(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff) - 1023;
    const unsigned long long m = u & 0xfffffffffffffULL;
    if (e < -126) return df{__uint_as_float(sign), 0.f};
    if (e > 127) return df{__uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u)), 0.f};
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    const unsigned r = (unsigned)(m & 0x1fffffffULL);
    float lo = 0.f;
    if (r != 0u) {
        // r 2^(e-52) by power-of-two factors that are normal FP32 numbers: the
        // first product is exact, the second rounds once into the subnormals
        const int sc = e - 52;
        const float rf = __uint2float_rn(r);
        lo = sc >= -126 ? rf * __uint_as_float((unsigned)(sc + 127) << 23)
                        : (rf * __uint_as_float((unsigned)(sc + 64 + 127) << 23)) * 5.421010862427522e-20f;  // 2^-64
        lo = __uint_as_float(__float_as_uint(lo) | sign);
    }
    return df{hi, lo};
}

// the double with the value of a normal (or zero, inf, nan) float, built from its fields
__device__ __forceinline__ double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned long long s = (unsigned long long)(b >> 31) << 63;
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned long long mant = (unsigned long long)(b & 0x7fffffu) << 29;
    if (ex == 0u) return __longlong_as_double((long long)s);
    if (ex == 0xffu) return __longlong_as_double((long long)(s | 0x7ff0000000000000ULL | mant));
    return __longlong_as_double((long long)(s | ((unsigned long long)(ex - 127u + 1023u) << 52) | mant));
}

__device__ __forceinline__ double join_df(df a) { return widen(a.hi) + widen(a.lo); }

}  // namespace ftcj
