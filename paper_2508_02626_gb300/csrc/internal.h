// internal.h -- structures shared by the host runtime (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dafmm.h"

namespace dafmm {

constexpr int kMaxOrder = DAFMM_MAX_ORDER;
constexpr int kQBits = 21;      // integer coordinate bits per axis (box membership)
constexpr int kMaxUniformDepth = 7;
constexpr int kNumKeys = 343;   // displacements v in [-3,3]^3; key = (vx+3)*49 + (vy+3)*7 + (vz+3)

__host__ __device__ constexpr int ncoef_of(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
// row stride of every expansion array: ncoef rounded up to 8 (32-byte rows in FP32)
__host__ __device__ constexpr int ncp_of(int p) { return (ncoef_of(p) + 7) / 8 * 8; }

// Harmonic basis.  The multipole expansions of 1/r are polynomials in d = r / r^2 whose
// homogeneous parts are solid harmonics (Eq. 2 is the generating function of the Legendre
// polynomials: its degree-n part is |s|^n |d|^n P_n(cos gamma)), and the local expansions are
// Taylor polynomials of a harmonic potential, whose homogeneous parts are harmonic too.  A
// harmonic homogeneous polynomial of degree n is fixed by its 2n + 1 coefficients with z
// exponent c <= 1: Laplace's equation gives every other one,
//   (c + 2)(c + 1) a[a, b, c + 2] = -(a + 2)(a + 1) a[a + 2, b, c] - (b + 2)(b + 1) a[a, b + 2, c],
// so an expansion of order p has (p + 1)^2 free coefficients instead of ncoef(p).
__host__ __device__ constexpr int nharm_of(int p) { return (p + 1) * (p + 1); }
// row stride of arrays of free coefficients: nharm rounded up to 8
__host__ __device__ constexpr int harm_row(int p) { return (nharm_of(p) + 7) / 8 * 8; }
// the coefficient index (the layout of da_index: degree, x exponent descending, y descending)
// of free coefficient k: degree n with n^2 <= k < (n + 1)^2, then within the degree the c <= 1
// coefficients in layout order: (n, 0, 0), (n - 1, 1, 0), (n - 1, 0, 1), (n - 2, 2, 0), ...
__host__ __device__ inline int harm_full_index(int k) {
    int n = 0;
    while ((n + 1) * (n + 1) <= k) ++n;
    const int r = k - n * n;
    const int a = n - (r + 1) / 2, c = (r > 0 && (r & 1) == 0) ? 1 : 0, b = n - a - c;
    return n * (n + 1) * (n + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

// ---- views passed by value to kernels ---------------------------------------------------
struct TreeView {
    int64_t n;
    int depth;        // uniform tree depth L (leaves at level L)
    int nleaf;        // 8^L
    double x0, y0, z0, size;
    double h_leaf, inv_h_leaf;
    const double *x, *y, *z, *q;  // sorted by leaf, FP64
    const float4* xq;             // leaf-scaled offsets (x - c)/h and charge, FP32, pair-interleaved
                                  // records from xq_base(leaf_start[l], l) per leaf l
                                  // and, xq_records(n, nleaf) float4s further, the FP32
                                  // remainders of those offsets (same records)
    const int* perm;              // sorted position -> input index
    const int* leaf_start;        // nleaf + 1
    int locals_f32;               // the leaf locals passed to the leaf kernel are FP32 rows
};

struct ShiftTab {                 // compressed rows of a level-independent M2M or L2L table
    const int* rowptr;
    const unsigned short* col;
    const unsigned char* par;     // bit v: exponent sum of row and column odd in axis v
    const double* val;
    const float* valf;
    const int* rp8;               // [nc * 8 + 1]: start of the entries of (row, parity class)
};

struct MulTab {                   // DA product table for the K generation
    const int* rowptr;            // per output coefficient k
    const ushort2* pairs;         // (i, j) with e_i + e_j = e_k
    const short* minus;           // [3][nc]: index of e_k - e_v, or -1
};

struct AdaptiveView;

// ---- per-order operator tables and launchers ------------------------------------------
struct OrderData {
    int p = -1, nc = 0, ncp = 0;
    int* m2m_rowptr = nullptr; unsigned short* m2m_col = nullptr; unsigned char* m2m_par = nullptr;
    double* m2m_val = nullptr; float* m2m_valf = nullptr;
    int* l2l_rowptr = nullptr; unsigned short* l2l_col = nullptr; unsigned char* l2l_par = nullptr;
    double* l2l_val = nullptr; float* l2l_valf = nullptr;
    int* m2m_rp8 = nullptr; int* l2l_rp8 = nullptr;
    // the M2M of harmonic multipoles (free rows composed with the expansion from the free
    // coefficients; no rp8 runs)
    int* m2mh_rowptr = nullptr; unsigned short* m2mh_col = nullptr; unsigned char* m2mh_par = nullptr;
    double* m2mh_val = nullptr; float* m2mh_valf = nullptr;
    // F16 splits of the M2L matrices with their power-of-two row and matrix factors
    void* Kh16 = nullptr; void* Kl16 = nullptr;
    float* k16_inv_r = nullptr; float* k16_inv_c = nullptr;
    // the same for the M2L in the harmonic basis: [343][npt_h][rowlen_h] F16 parts of
    // K^_v restricted to the free coefficients (rows) and composed with the expansion from them
    // (columns), and the expansion's steps (harm_expand_launch)
    void* Kh16h = nullptr; void* Kl16h = nullptr;
    float* k16h_inv_r = nullptr; float* k16h_inv_c = nullptr;
    float* Khih = nullptr; float* Kloh = nullptr;  // TF32 parts [343][npt_h][harm_row] (MIXED)
    int4* hx_step = nullptr;      // [ncoef - nharm]: (i, i1, i2, 0), in order of increasing c
    float2* hx_w = nullptr;       // their weights (w1, w2): a[i] = w1 a[i1] + w2 a[i2]
    double2* hx_w64 = nullptr;    // the same weights in FP64 (the multipoles' fill)
    int hx_cst[kMaxOrder + 3] = {};  // steps of z exponent c: [hx_cst[c], hx_cst[c + 1])
    int* mul_rowptr = nullptr; ushort2* mul_pairs = nullptr; short* mul_minus = nullptr;
    size_t mul_npairs = 0;
    double* K64 = nullptr;        // [343][nc][ncp]: K^_v[b][a] (scaled M2L, Eq. 5)
    float* K32 = nullptr;         // same in FP32
    float* Khi = nullptr;         // [343][npt][ncp] TF32 high / low parts for the tensor-core M2L
    float* Klo = nullptr;
    float* M2Mhi = nullptr;       // [8][npt][ncp] dense M2M / L2L tables per child octant, TF32 parts
    float* M2Mlo = nullptr;
    float* L2Lhi = nullptr;
    float* L2Llo = nullptr;
    bool k_ready = false;
    // M2L by rotation (Sec. 3.4): per key the four substitution tables, per key the index of
    // its axial length, the axial matrices' structural non-zeros (CSR by row) per length
    double* rot_T = nullptr;
    int* rot_rho = nullptr;
    int* ax_rowptr = nullptr;
    unsigned short* ax_col = nullptr;
    double* ax_val = nullptr;
    int ax_nnz = 0, n_rho = 0;
    // the kernel's load-balanced task lists (x-step, z-step, axial), [length][32] each
    uint2* rot_lx = nullptr;
    uint2* rot_lz = nullptr;
    uint2* rot_la = nullptr;
    int rot_len[3] = {0, 0, 0};
    // the same lists in the harmonic form (outputs of z exponent <= 1 only) and the steps that
    // restore the other coefficients (FP64 weights; harm_steps in api.cu)
    uint2* rot_lxh = nullptr;
    uint2* rot_lzh = nullptr;
    uint2* rot_lah = nullptr;
    int rot_lenh[3] = {0, 0, 0};
    int4* hxr_step = nullptr;
    double2* hxr_w = nullptr;
    int hxr_cst[kMaxOrder + 3] = {};
    // float-float copies of rot_T and ax_val (the DAFMM_FF mode's M2L), made on first use
    float2* rot_Tf = nullptr;
    float2* ax_valf = nullptr;
    ShiftTab m2m() const { return ShiftTab{m2m_rowptr, m2m_col, m2m_par, m2m_val, m2m_valf, m2m_rp8}; }
    ShiftTab l2l() const { return ShiftTab{l2l_rowptr, l2l_col, l2l_par, l2l_val, l2l_valf, l2l_rp8}; }
    ShiftTab m2mh() const { return ShiftTab{m2mh_rowptr, m2mh_col, m2mh_par, m2mh_val, m2mh_valf, nullptr}; }
    MulTab mul() const { return MulTab{mul_rowptr, mul_pairs, mul_minus}; }
};

// host copies of the generated tables (generated/da_tables_p*.h), per order
struct HostShiftTable {
    int nnz;
    const int* rowptr;
    const unsigned short* col;
    const unsigned char* par;     // non-decreasing within each row
    const double* val;
};

// starts of the (row, parity class) runs of a shift table: out[8 * b + m] for m = 0..7, and
// out[8 * nc] = nnz
inline void shift_rp8(const HostShiftTable& t, int nc, int* out) {
    for (int b = 0; b < nc; ++b) {
        int e = t.rowptr[b];
        for (int m = 0; m < 8; ++m) {
            while (e < t.rowptr[b + 1] && t.par[e] < m) ++e;
            out[8 * b + m] = e;
        }
    }
    out[8 * nc] = t.nnz;
}

// or-ed into the precision argument of p2m and m2m_level (FP32 mode only): the multipole
// rows are FP32 (ncp floats per box, in the FP64 arrays' memory) instead of FP64
constexpr int kRowsF32 = 0x100;
// or-ed into the precision argument of m2l_a (FP64 only): the M2L by rotation (Sec. 3.4)
constexpr int kM2LRot = 0x200;
constexpr int kM2LHarm = 0x400;  // with kM2LRot: the rotation in its harmonic form
// or-ed into the precision argument of p2m, m2m_level, p2m_a and m2m_a (FP32 and MIXED): the
// multipoles are harmonic-basis rows -- only the (p + 1)^2 free coefficients (z exponent <= 1)
// are computed and written, at their layout positions; the other entries are left as they are
// (adaptive trees fill them in afterwards, tc_harm_fill, for the M2P)
constexpr int kRowsHarm = 0x800;

// F16 split rows written by the P2M itself (the FP32 mode's harmonic basis, finest level): row
// b of hi and lo holds rowlen halves (the free coefficients scaled by 2^-e, e the exponent of
// the row's largest magnitude, zero-padded), inv[b] = 2^e -- what tc_split_f16_multi writes
struct F16Rows {
    void* hi = nullptr;
    void* lo = nullptr;
    float* inv = nullptr;
    int rowlen = 0;
};

struct OrderOps {
    int p, nc, ncp;
    HostShiftTable m2m, l2l, m2mh;
    // precision argument: DAFMM_FP64 / DAFMM_MIXED / DAFMM_FP32
    // f16 (optional, FP32 harmonic rows only): the F16 split of the rows, written as well
    cudaError_t (*p2m)(const TreeView&, int prec, double* Mleaf, const F16Rows* f16, cudaStream_t);
    cudaError_t (*m2m_level)(const OrderData&, int prec, int lchild, const double* Mc, double* Mp,
                             cudaStream_t);
    cudaError_t (*l2l_level)(const OrderData&, int prec, int lchild, const double* Lp, double* Lc,
                             cudaStream_t);
    cudaError_t (*m2l_level)(const OrderData&, int prec, int level, const double* M, const float* Mf,
                             double* L, double inv_h, cudaStream_t);
    cudaError_t (*leaf)(const TreeView&, int prec, const double* Lleaf, double* phi, double* field,
                        cudaStream_t);
    cudaError_t (*kgen)(OrderData&, const short* key_list, int nkeys, cudaStream_t);  // null list: all keys
    // M2L by rotation (FP64) of a uniform tree's level, and its tables (adaptive trees: m2l_a
    // with kM2LRot)
    cudaError_t (*m2l_rot)(const OrderData&, int level, const double* M, double* L, double inv_h, bool harm,
                           cudaStream_t);
    cudaError_t (*rot_setup)(OrderData&, const double* r0s, int nrho, double* Kscratch, cudaStream_t);
    int rot_tsz;  // doubles per substitution table (sum over m <= p of (m+1)^2)
    cudaError_t (*op_p2m)(int prec, int64_t n, const double* s, const double* q, double* out, cudaStream_t);
    cudaError_t (*op_p2l)(int prec, int64_t n, const double* w, const double* q, double* out, cudaStream_t);
    cudaError_t (*op_l2p)(int prec, int64_t n, const double* L, const double* x, double* out4, cudaStream_t);
    cudaError_t (*op_m2p)(int prec, int64_t n, const double* M, const double* s, double* out4, cudaStream_t);
    cudaError_t (*op_shift)(const OrderData&, int which, int prec, int64_t n, const int* oct,
                            const double* in, double* out, cudaStream_t);
    // adaptive trees
    cudaError_t (*p2m_a)(const AdaptiveView&, const int* leaves, int nleaves, int prec, double* M, cudaStream_t);
    cudaError_t (*m2m_a)(const OrderData&, const AdaptiveView&, int prec, int lb, int le, double* M, cudaStream_t);
    cudaError_t (*m2l_a)(const OrderData&, const AdaptiveView&, int prec, const int* tg, const int* grp_ptr, int grp0,
                         int max_group, const double* M, const float* Mf, double* L, cudaStream_t);
    cudaError_t (*p2l_a)(const AdaptiveView&, int prec, int lb, int le, double* L, cudaStream_t);
    // L2L from the parents [lb, le) of one level into their children
    cudaError_t (*l2l_a)(const OrderData&, const AdaptiveView&, int prec, int lb, int le, double* L, cudaStream_t);
    cudaError_t (*leaf_a)(const AdaptiveView&, const int* leaves, int nleaves, int prec, const double* L,
                          const double* M, const float* Mf, double* phi, double* field, int warps, cudaStream_t);
    // the M2L by rotation of a uniform tree's level in float-float (DAFMM_FF; tables rot_Tf,
    // ax_valf; source rows as FP32 high and low parts), and the conversion of n doubles into
    // float-float pairs
    cudaError_t (*m2l_rot_ff)(const OrderData&, int level, const float* Mh, const float* Ml, double* L, double inv_h,
                              bool harm, cudaStream_t);
    cudaError_t (*to_ff)(const double* a, float2* b, size_t n, cudaStream_t);
    // the float-float split of n FP64 values into their FP32 high and low parts
    cudaError_t (*split_ff)(const double* a, float* hi, float* lo, size_t n, cudaStream_t);
};

const OrderOps* order_ops(int p);

// harm_fill.cu: the coefficients of z exponent >= 2 of nrows FP64 multipole rows (ncp doubles
// each) from their free ones, in place; step, w and cst as made by the harmonic-basis setup
// (OrderData::hx_step, hx_w64, hx_cst)
cudaError_t harm_fill(int p, double* M, int nrows, const int4* step, const double2* w, const int* cst, cudaStream_t s);

// numerical-DA operator batches (da_numeric.cu), FP64, one warp per instance; `op` is one of
// kDa*, the arguments those of the single-operator entry points (a: first array, b: second,
// oct: child octants of M2M/L2L)
enum { kDaP2M = 0, kDaP2L, kDaL2P, kDaM2P, kDaM2M, kDaL2L, kDaM2L };
cudaError_t launch_da_op(const OrderData& od, int op, int64_t n, const double* a, const double* b, const int* oct,
                         double* out, int num_sms, cudaStream_t s);
// one function per translation unit fmm_p*.cu
#define DAFMM_DECLARE_ORDER(P) const OrderOps* order_ops_p##P();
DAFMM_DECLARE_ORDER(0) DAFMM_DECLARE_ORDER(1) DAFMM_DECLARE_ORDER(2) DAFMM_DECLARE_ORDER(3)
DAFMM_DECLARE_ORDER(4) DAFMM_DECLARE_ORDER(5) DAFMM_DECLARE_ORDER(6) DAFMM_DECLARE_ORDER(7)
DAFMM_DECLARE_ORDER(8) DAFMM_DECLARE_ORDER(9) DAFMM_DECLARE_ORDER(10)
#undef DAFMM_DECLARE_ORDER

// ---- tree build (tree_build.cu) ---------------------------------------------------------
// device min/max of the coordinates: out6 = {xmin, ymin, zmin, xmax, ymax, zmax} (device)
cudaError_t launch_bbox(const double* xyz, int64_t n, double* out6, cudaStream_t s);
// leaf keys of a uniform tree and identity values
cudaError_t launch_uniform_keys(const double* xyz, int64_t n, double x0, double y0, double z0,
                                double scale, int depth, uint64_t* keys, int* vals, cudaStream_t s);
// stable LSD radix sort of (key, value) pairs on the low `bits` bits of the key
size_t radix_sort_temp_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint64_t* keys, int* vals, int64_t n, int bits, void* temp,
                             cudaStream_t s);
// gather sorted SoA arrays and leaf-scaled FP32 copies; leaf ranges by binary search
cudaError_t launch_gather_uniform(const double* xyz, const double* q, const int* perm, int64_t n,
                                  const uint64_t* sorted_keys, TreeView tv, double* x, double* y,
                                  double* z, double* qs, float4* xq, int* leaf_start,
                                  cudaStream_t s);
cudaError_t launch_scatter_outputs(const double* phi_sorted, const double* field_sorted, const int* perm,
                                   int64_t n, double* phi, double* field, cudaStream_t s);

}  // namespace dafmm
