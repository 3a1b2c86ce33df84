// m2l_tc.h -- host interface of the tensor-core M2L (m2l_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "internal.h"

namespace dafmm {

constexpr int kTcMaxLevels = kMaxUniformDepth - 1;  // levels 2..7

// kernel parameters (passed as a __grid_constant__ struct; tensor maps are 64-byte aligned)
struct M2LTCParams {
    CUtensorMap a_hi[kTcMaxLevels];
    CUtensorMap a_lo[kTcMaxLevels];
    CUtensorMap b_hi;
    CUtensorMap b_lo;
    double* L[kTcMaxLevels];
    double inv_h[kTcMaxLevels];
    int P[kTcMaxLevels];
    int bx[kTcMaxLevels], by[kTcMaxLevels], bz[kTcMaxLevels];
    int tile_base[kTcMaxLevels + 1];
    int nlev;
    int ntiles;
    int nhalf;
    int* err;
};

struct M2LTCArgs {
    int lmin, lmax;                              // levels with M2L work (2..depth)
    const float* Mhi[kMaxUniformDepth + 1];      // per level, [8^l][ncp], TF32 high part
    const float* Mlo[kMaxUniformDepth + 1];      // TF32 low part
    double* L[kMaxUniformDepth + 1];             // per level outputs (written, not added)
    double inv_h[kMaxUniformDepth + 1];
    const float* Khi;                            // [343][npt][ncp]
    const float* Klo;
    int* err;                                    // device error flag
    int num_sms;
};

int m2l_tc_npt(int p);  // rows of the split K^ tables (nc padded to the MMA N granule)
cudaError_t m2l_tc_split_tf32(const double* src, float* hi, float* lo, size_t n, cudaStream_t s);
cudaError_t m2l_tc_split_k(const double* K64, int p, float* hi, float* lo, cudaStream_t s);
cudaError_t m2l_tc_launch(int p, const M2LTCArgs& a, cudaStream_t s);

}  // namespace dafmm
