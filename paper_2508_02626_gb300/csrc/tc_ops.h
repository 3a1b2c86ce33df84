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
    // F16 operands only: per-box factors of the A rows (per level), per-column and per-matrix
    // factors of the B matrices (see tc_split_f16 / tc_prepare_k16)
    const float* a_inv[kTcMaxLevels];
    const float* inv_r;
    const float* inv_c;
    int nlev;
    int ntiles;
    int nhalf;
    int mode;
    int out_f32;  // out rows hold FP32 values (NCP floats per box) instead of FP64
    int* err;
};

// one launch: M2L over levels lmin..lmax, or one M2M / L2L level (lmin = lmax = child level)
struct TCArgs {
    int mode;
    int lmin, lmax;
    bool f16;                                    // F16 split operands (M2L only), else TF32
    bool harm;                                   // (M2L) the harmonic basis: A rows, matrices
                                                 // and out rows hold the free coefficients only
    const void* a_hi[kMaxUniformDepth + 1];      // per level, [8^l][rowlen] split parts of the A operand
    const void* a_lo[kMaxUniformDepth + 1];
    const float* a_inv[kMaxUniformDepth + 1];    // F16: per-box factor undoing the row scale
    double* out[kMaxUniformDepth + 1];           // FP64 result per level (written; added for L2L)
    bool out_f32;                                // out rows hold FP32 values instead (NCP floats per box)
    float* out_hi[kMaxUniformDepth + 1];         // optional TF32 split of the result
    float* out_lo[kMaxUniformDepth + 1];
    double scale[kMaxUniformDepth + 1];
    const void* b_hi;                            // [nkey][npt][rowlen] split parts of the matrices
    const void* b_lo;
    const float* inv_r;                          // F16: per-column factor of the matrices
    const float* inv_c;                          // F16: per-matrix factor
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
    const void* a_hi;         // [nbox][rowlen] split parts of the multipoles (TF32 or F16)
    const void* a_lo;
    const float* a_inv;       // F16: per-box factor undoing the row scale
    const float* inv_r;       // F16: per-column factor of the matrices
    const float* inv_c;       // F16: per-matrix factor
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
#if defined(DAFMM_CHECK)
    int nbox;                 // checked builds: boxes (the bound of the index checks)
#endif
};

struct TCGArgs {
    bool f16;
    bool harm;                // the harmonic basis: A rows and matrices hold the free
                              // coefficients; out receives FP32 rows of them (harm_row(p) floats)
    const void* a_hi;
    const void* a_lo;
    const float* a_inv;
    const void* b_hi;         // [nkey][npt][rowlen] split parts of the M2L matrices
    const void* b_lo;
    const float* inv_r;
    const float* inv_c;
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
    int nbox;                 // boxes of the tree (the bound of the checked build's index checks)
};


int tc_npt(int p);  // rows of the split matrix tables (nc padded to the MMA N granule)
int tc_rowlen16(int p);  // F16 operand row length: ncoef rounded up to 16
// F16 split of FP64 rows [nrows][ncp] with a power-of-two scale per row (row max in [0.5, 1)):
// hi, lo [nrows][rowlen16] halves, inv[nrows] = the factor that undoes the scale
cudaError_t tc_split_f16(const double* src, int nrows, int p, void* hi, void* lo, float* inv, cudaStream_t s);
// the same for up to 8 arrays in one launch; src_f32: the rows are FP32 (ncp floats per row);
// harm: only the free coefficients of the harmonic basis, into rows of tc_rowlen16h(p) halves
cudaError_t tc_split_f16_multi(int nseg, const void* const* src, const int* nrows, void* const* hi, void* const* lo,
                               float* const* inv, int p, cudaStream_t s, bool src_f32, bool harm);
// F16 split of the M2L matrices K[nkey][nc][ncp] (FP64): row b of matrix k is scaled by
// r_b c_k (powers of two: r_b from the largest entry of row b over all matrices, c_k from the
// largest entry of the row-scaled matrix k); hi, lo [nkey][npt][rowlen16]; inv_r[npt],
// inv_c[nkey] undo the scales.  `scratch` holds nkey + npt floats.
cudaError_t tc_prepare_k16(const double* K, int nkey, int p, void* hi, void* lo, float* inv_r, float* inv_c,
                           float* scratch, cudaStream_t s);
// The M2L in the harmonic basis (nharm_of(p) free coefficients, harm_full_index): npt / rowlen
// of its matrix tables, and the tables: Kh = K restricted to the free output coefficients and
// composed with X [nc][nh] (the expansion from the free input coefficients), as FP64 scratch
// [nkey][nh][nhp = nh rounded up to 8], then split as tc_prepare_k16 does (scratch: npt + nkey
// floats); thi / tlo receive the TF32 parts of Kh as [nkey][npt][nhp] (the MIXED mode's form).
int tc_npt_h(int p);
int tc_rowlen16h(int p);
cudaError_t tc_prepare_k16h(const double* K, int nkey, int p, const double* X, double* Kh, void* hi, void* lo,
                            float* inv_r, float* inv_c, float* scratch, float* thi, float* tlo, cudaStream_t s);
// TF32 parts of the free coefficients of FP64 rows [nrows][ncp]: hi, lo [nrows][harm_row(p)]
cudaError_t tc_split_tf32_harm(const double* src, size_t nrows, int p, float* hi, float* lo, cudaStream_t s);
// rows of free coefficients (FP32, nhp per row) of up to kTcMaxLevels arrays -> full rows (FP32
// or FP64, ncp per row) by Laplace's equation: steps (i, i1, i2) with weights (w1, w2), those of
// z exponent c at [cst[c], cst[c + 1]); hi / lo (optional, per array or null) receive the TF32
// split of the written rows
cudaError_t tc_harm_expand(int p, int nseg, const float* const* red, void* const* full, float* const* hi,
                           float* const* lo, const int* nrows, bool full_f32, const int4* step, const float2* w,
                           const int* cst, cudaStream_t s);
cudaError_t tcg_launch(int p, const TCGArgs& a, cudaStream_t s);
cudaError_t tc_split_tf32(const double* src, float* hi, float* lo, size_t n, cudaStream_t s);
cudaError_t tc_split_rows(const double* src, int nkey, int p, float* hi, float* lo, cudaStream_t s);
cudaError_t tc_launch(int p, const TCArgs& a, cudaStream_t s);

}  // namespace dafmm
