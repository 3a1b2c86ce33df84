// tc_ops.h -- host interface of the tensor-core contractions (tc_ops.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "internal.h"

namespace dafmm {

constexpr int kTcMaxLevels = kMaxUniformDepth - 1;  // levels 2..7
constexpr int kTcM2L = 0, kTcM2M = 1, kTcL2L = 2;

// kernel parameters (passed as a __grid_constant__ struct; tensor maps are 64-byte aligned)
struct TCParams {
    CUtensorMap a_hi[kTcMaxLevels];
    CUtensorMap a_lo[kTcMaxLevels];
    CUtensorMap b_hi;
    CUtensorMap b_lo;
    double* out[kTcMaxLevels];
    float* out_hi[kTcMaxLevels];
    float* out_lo[kTcMaxLevels];
    double scale[kTcMaxLevels];
    int S[kTcMaxLevels];
    int bx[kTcMaxLevels], by[kTcMaxLevels], bz[kTcMaxLevels];
    int out_level[kTcMaxLevels];
    int tile_base[kTcMaxLevels + 1];
    int nlev;
    int ntiles;
    int nhalf;
    int mode;
    int* err;
};

// one launch: M2L over levels lmin..lmax, or one M2M / L2L level (lmin = lmax = child level)
struct TCArgs {
    int mode;
    int lmin, lmax;
    const float* a_hi[kMaxUniformDepth + 1];     // per level, [8^l][ncp] TF32 parts of the A operand
    const float* a_lo[kMaxUniformDepth + 1];
    double* out[kMaxUniformDepth + 1];           // FP64 result per level (written; added for L2L)
    float* out_hi[kMaxUniformDepth + 1];         // optional TF32 split of the result
    float* out_lo[kMaxUniformDepth + 1];
    double scale[kMaxUniformDepth + 1];
    const float* b_hi;                           // [nkey][npt][ncp] TF32 parts of the matrices
    const float* b_lo;
    int nkey;
    int* err;                                    // device error flag
    int num_sms;
};

// ---- gathered form (adaptive trees and forests) ----
// Targets come in groups (boxes of one level and octant, contiguous in `tg`); the A rows of a
// tile of 128 targets are gathered row by row, so any tree shape works.
constexpr int kTcgMaxGroups = 8 * 21;  // (level, octant) groups of a launch

struct TCGParams {
    CUtensorMap b_hi;
    CUtensorMap b_lo;
    const float* a_hi;        // [nbox][ncp] TF32 parts of the multipoles
    const float* a_lo;
    const int* tg;            // target boxes, grouped
    const int* parent;
    const int* colleague;     // 27 per box
    const int* child;         // 8 per box
    const double4* geom;      // per box: centre and width (scale 1/width)
    double* out;              // [nbox][ncp], written
    // work groups in launch order: octant-major (the CTAs running at the same time share one
    // octant's 189 matrices in L2), then level; within a group tile-major with the output
    // halves of a tile next to each other (they gather the same source rows)
    int grp_start[kTcgMaxGroups];
    int grp_count[kTcgMaxGroups];
    int grp_oct[kTcgMaxGroups];
    int tile_base[kTcgMaxGroups + 1];
    int ngroups;
    int ntiles;
    int nhalf;
    int* err;
};

struct TCGArgs {
    const float* a_hi;
    const float* a_lo;
    const float* b_hi;        // [nkey][npt][ncp] TF32 parts of the M2L matrices
    const float* b_lo;
    int nkey;
    const int* tg;
    const int* parent;
    const int* colleague;
    const int* child;
    const double4* geom;
    double* out;
    int ngroups;
    int grp_start[kTcgMaxGroups];
    int grp_count[kTcgMaxGroups];
    int grp_oct[kTcgMaxGroups];
    int* err;
    int num_sms;
};

int tc_npt(int p);  // rows of the split matrix tables (nc padded to the MMA N granule)
cudaError_t tcg_launch(int p, const TCGArgs& a, cudaStream_t s);
cudaError_t tc_split_tf32(const double* src, float* hi, float* lo, size_t n, cudaStream_t s);
cudaError_t tc_split_rows(const double* src, int nkey, int p, float* hi, float* lo, cudaStream_t s);
cudaError_t tc_launch(int p, const TCArgs& a, cudaStream_t s);

}  // namespace dafmm
