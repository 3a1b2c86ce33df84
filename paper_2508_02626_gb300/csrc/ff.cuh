// ff.cuh -- float-float numbers: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits, computed on the FP32 pipe.  On this part the
// FP32 FMA rate is about 70 times the FP64 one, so float-float arithmetic (7 to 15 FP32
// instructions per operation) carries FP64-level accuracy several times faster than FP64.
//
// Built from the error-free transformations TwoSum (Knuth: s + e = a + b exactly), Fast2Sum
// (Dekker: the same when |a| >= |b| or a = 0) and TwoProd by FMA (p + e = a b exactly), with the
// double-word algorithms of Joldes, Muller and Popescu (ACM TOMS 43, 2017): the sum of two
// double-words (their "accurate" DWPlusDW, relative error below 3 u^2 for u = 2^-24) and the
// product (DWTimesDW, below 5 u^2).  1/sqrt takes the FP32 approximation and one Newton step with
// its residual in float-float (relative error about u^2 times a small constant).  The exponent
// range is FP32's: values far from 1 (beyond about 2^+-100) lose low bits of lo to underflow.
//
// The operators let the generated straight-line operators, written for a type T, run in
// float-float (T(constant) splits a double constant into hi + lo).
#pragma once
#include <math.h>

#include "da_common.cuh"

namespace dafmm {

// an FP32 product that the compiler never fuses with a following addition (a fused one would
// break the exactness the transformations below rely on)
DAFMM_HD DAFMM_INLINE float mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

// FP32 seeds of 1/sqrt(x) and 1/x for one Newton step (the step supplies the accuracy): the
// hardware approximations on the GPU (relative error a few 2^-23), IEEE FP32 on the host
DAFMM_HD DAFMM_INLINE float rsqrt_seed(float x) {
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}
DAFMM_HD DAFMM_INLINE float rcp_seed(float x) {
#if defined(__CUDA_ARCH__)
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}

struct ff {
    float hi, lo;
    ff() = default;
    DAFMM_HD constexpr ff(float h, float l) : hi(h), lo(l) {}
    DAFMM_HD explicit ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    DAFMM_HD explicit ff(int i) : ff((double)i) {}
    DAFMM_HD double to_double() const { return (double)hi + (double)lo; }
    DAFMM_HD explicit operator double() const { return (double)hi + (double)lo; }
    DAFMM_HD explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (TwoSum)
DAFMM_HD DAFMM_INLINE ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return ff(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Fast2Sum)
DAFMM_HD DAFMM_INLINE ff fast_two_sum(float a, float b) {
    const float s = a + b;
    return ff(s, b - (s - a));
}
// p + e = a b exactly (TwoProd by FMA)
DAFMM_HD DAFMM_INLINE ff two_prod(float a, float b) {
    const float p = mul_rn(a, b);
    return ff(p, fmaf(a, b, -p));
}

// x + y (accurate DWPlusDW)
DAFMM_HD DAFMM_INLINE ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    const ff t = two_sum(x.lo, y.lo);
    const ff v = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(v.hi, v.lo + t.lo);
}
// x + y for running sums (sloppy DWPlusDW: error below 2 u^2 (|x| + |y|), relative to the
// terms rather than to the sum -- as an FP64 sum's; 10 instead of 20 instructions)
DAFMM_HD DAFMM_INLINE ff ff_acc(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
// x y (DWTimesDW)
DAFMM_HD DAFMM_INLINE ff ff_mul(ff x, ff y) {
    const ff c = two_prod(x.hi, y.hi);
    const float tl = fmaf(x.hi, y.lo, mul_rn(x.lo, y.hi));
    return fast_two_sum(c.hi, c.lo + tl);
}
// x times an FP32 number
DAFMM_HD DAFMM_INLINE ff ff_mul(ff x, float y) {
    const ff c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, fmaf(x.lo, y, c.lo));
}
DAFMM_HD DAFMM_INLINE ff ff_neg(ff x) { return ff(-x.hi, -x.lo); }

// 1/sqrt(x) for x > 0: y = an FP32 seed of 1/sqrt(x.hi), then one Newton step
// y' = y + y (1 - x y^2) / 2, the residual 1 - x y^2 computed in float-float (the seed's error
// e becomes about 3 e^2 / 2 + u^2)
DAFMM_HD DAFMM_INLINE ff ff_rsqrt(ff x) {
    const float y = rsqrt_seed(x.hi);
    const ff r = ff_add(ff(1.0f, 0.0f), ff_neg(ff_mul(x, ff_mul(ff(y, 0.0f), y))));
    return fast_two_sum(y, mul_rn(0.5f * y, r.hi));
}
// 1/x: y = an FP32 seed of 1/x.hi, then y' = y + y (1 - x y) (error about e^2 + u^2)
DAFMM_HD DAFMM_INLINE ff ff_rcp(ff x) {
    const float y = rcp_seed(x.hi);
    const ff r = ff_add(ff(1.0f, 0.0f), ff_neg(ff_mul(x, y)));
    return fast_two_sum(y, mul_rn(y, r.hi));
}

DAFMM_HD DAFMM_INLINE ff operator+(ff a, ff b) { return ff_add(a, b); }
DAFMM_HD DAFMM_INLINE ff operator-(ff a, ff b) { return ff_add(a, ff_neg(b)); }
DAFMM_HD DAFMM_INLINE ff operator-(ff a) { return ff_neg(a); }
DAFMM_HD DAFMM_INLINE ff operator*(ff a, ff b) { return ff_mul(a, b); }
DAFMM_HD DAFMM_INLINE ff& operator+=(ff& a, ff b) { return a = ff_add(a, b); }
DAFMM_HD DAFMM_INLINE ff& operator-=(ff& a, ff b) { return a = ff_add(a, ff_neg(b)); }
DAFMM_HD DAFMM_INLINE ff& operator*=(ff& a, ff b) { return a = ff_mul(a, b); }

// the functions the generated operators call
DAFMM_HD DAFMM_INLINE ff dafmm_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }
DAFMM_HD DAFMM_INLINE ff dafmm_rsqrt(ff x) { return ff_rsqrt(x); }
DAFMM_HD DAFMM_INLINE ff dafmm_rcp(ff x) { return ff_rcp(x); }
DAFMM_HD DAFMM_INLINE ff dafmm_sqrt(ff x) { return ff_mul(x, ff_rsqrt(x)); }

}  // namespace dafmm
