// da_common.cuh -- helpers shared by the generated DA-FMM operators and the kernels.
//
// The generated operator code (generated/da_ops_p*.cuh) is plain arithmetic on a
// template type T (float or double) and compiles both for the GPU (nvcc) and for
// the host (g++), so that the host build can be checked without a GPU.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define DAFMM_HD __host__ __device__
#define DAFMM_INLINE __forceinline__
#else
#define DAFMM_HD
#define DAFMM_INLINE inline
#endif

namespace dafmm {

// number of DA coefficients of order p in three variables: C(p+3, 3)
DAFMM_HD constexpr int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// coefficient index of d1^a d2^b d3^c: graded by n = a+b+c, then x exponent
// descending, then y exponent descending (the order of the paper's Table 1)
DAFMM_HD constexpr int da_index(int a, int b, int c) {
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

DAFMM_HD DAFMM_INLINE double dafmm_fma(double a, double b, double c) { return fma(a, b, c); }
DAFMM_HD DAFMM_INLINE float dafmm_fma(float a, float b, float c) { return fmaf(a, b, c); }

DAFMM_HD DAFMM_INLINE double dafmm_rcp(double x) { return 1.0 / x; }
DAFMM_HD DAFMM_INLINE float dafmm_rcp(float x) { return 1.0f / x; }
DAFMM_HD DAFMM_INLINE double dafmm_sqrt(double x) { return sqrt(x); }
DAFMM_HD DAFMM_INLINE float dafmm_sqrt(float x) { return sqrtf(x); }

// 1/sqrt(x).  Double: CUDA's rsqrt() on the device, 1/sqrt on the host.
// Float on the device: the hardware approximation rsqrtf() refined by one
// Newton-Raphson step y <- y (3 - x y^2) / 2 (an FP32 seed plus one refinement).
DAFMM_HD DAFMM_INLINE double dafmm_rsqrt(double x) {
#if defined(__CUDA_ARCH__)
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}
DAFMM_HD DAFMM_INLINE float dafmm_rsqrt(float x) {
#if defined(__CUDA_ARCH__)
    float y = rsqrtf(x);
    return y * fmaf(-0.5f * x, y * y, 1.5f);
#else
    return 1.0f / sqrtf(x);
#endif
}

}  // namespace dafmm
