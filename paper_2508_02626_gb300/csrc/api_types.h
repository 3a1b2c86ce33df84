// api_types.h -- the opaque handles of the C ABI (contexts and trees), shared by the
// runtime translation units.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <string>
#include <utility>
#include <vector>

#include "internal.h"
#include "arena.h"
#include "tree_adaptive.h"

struct dafmm_ctx {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    std::string err;
    dafmm::OrderData ord[dafmm::kMaxOrder + 1];
    std::vector<dafmm_tree*> trees;
    // profiling: events at the phase boundaries of the last evaluation
    bool profile = false;
    cudaEvent_t ev[8] = {};
    cudaEvent_t ev_in = nullptr;  // end of a build's input copies (asynchronous uniform builds)
    int last_launches = 0;
    bool have_profile = false;
    int m2l_kernel = 0;       // 0 tensor cores, 1 SIMT
    int tc_mask = 5;          // FP32 mode: bit 0 M2L, bit 1 M2M, bit 2 L2L on the tensor cores
    int leaf_warps = 4;       // adaptive leaf kernel: leaves (one warp each) per thread block
    int m2l_f16 = 1;          // FP32 mode: M2L on F16 split operands (else TF32)
    int m2l_harm = 1;         // FP32 mode, uniform trees: the F16 M2L in the harmonic basis
    int m2l_rot = -1;         // FP64 mode: M2L by rotation (Sec. 3.4), uniform and adaptive; -1 = from p = 4
    int num_sms = 0;
    bool tc_capable = false;  // compute capability 10.x
    int* d_err = nullptr;     // device-side failure record of bounded waits
    // pooled contexts: every allocation comes from one reservation (no cudaFree, no device sync)
    char* arena_base = nullptr;
    dafmm::OffsetArena arena;
};

struct Expansions {
    int p = -1;
    int depth = -1;
    double* M[dafmm::kMaxUniformDepth + 1] = {};
    double* L[dafmm::kMaxUniformDepth + 1] = {};
    float* Mf[dafmm::kMaxUniformDepth + 1] = {};
    float* Mhi[dafmm::kMaxUniformDepth + 1] = {};
    float* Mlo[dafmm::kMaxUniformDepth + 1] = {};
    float* Lhi[dafmm::kMaxUniformDepth + 1] = {};
    float* Llo[dafmm::kMaxUniformDepth + 1] = {};
    // F16 splits of the multipoles (rows of ncoef rounded up to 16) and their row factors
    void* Mh16[dafmm::kMaxUniformDepth + 1] = {};
    void* Ml16[dafmm::kMaxUniformDepth + 1] = {};
    float* Minv[dafmm::kMaxUniformDepth + 1] = {};
    // the harmonic-basis M2L's output rows (free coefficients, FP32, nharm rounded up to 8)
    float* Lh[dafmm::kMaxUniformDepth + 1] = {};
    bool L_f32 = false;  // the last evaluation left FP32 rows (ncp floats per box) in L
    bool M_f32 = false;  // ... and in M
    bool M_harm = false;  // ... and harmonic-basis multipoles (free coefficients only) in M
};

struct dafmm_tree {
    dafmm_ctx* ctx = nullptr;
    int64_t n = 0;
    double dom[4] = {0, 0, 0, 1};
    int depth = 0;
    int nleaf = 1;
    int max_per_leaf = 0;           // -1: not read back yet (the asynchronous uniform build)
    double *x = nullptr, *y = nullptr, *z = nullptr, *q = nullptr;
    float4* xq = nullptr;  // 2 * xq_n4 float4s: FP32 records, then their remainders
    size_t xq_n4 = 0;      // float4s of one half of xq
    int* perm = nullptr;
    int* leaf_start = nullptr;
    Expansions ex;
    double* out_scratch = nullptr;  // device outputs when the caller passes host buffers
    size_t out_scratch_bytes = 0;
    // a uniform tree built asynchronously (pooled contexts): `built` completes with the build
    // on its stream; the build's scratch (`deferred`) goes back to the pool once it has
    cudaEvent_t built = nullptr;
    std::vector<std::pair<void*, size_t>> deferred;
    // adaptive trees (boxes breadth-first; see tree_adaptive.h)
    bool adaptive = false;
    int nbox = 1, maxlev = 0, cap = 0, max_leaf = 0;
    std::vector<int> level_start;   // first box of each level, plus the end
    int nroots = 1;                 // trees in the forest (one root box each)
    std::vector<double> rootdom;    // 4 per tree: x0, y0, z0, size
    std::vector<int64_t> root_offs; // particles of tree r: [root_offs[r], root_offs[r+1]) in input order
    double* d_rootdom = nullptr;
    double4* a_geom = nullptr;      // per box: centre and width
    int* a_xq0 = nullptr;           // per leaf box: its first FP32 record (even)
    int* a_root = nullptr;
    int *a_level = nullptr, *a_ijk = nullptr, *a_parent = nullptr, *a_child = nullptr;
    int *a_pbeg = nullptr, *a_pend = nullptr, *a_colleague = nullptr;
    int *u_ptr = nullptr, *u_idx = nullptr, *w_ptr = nullptr, *w_idx = nullptr, *x_ptr = nullptr, *x_idx = nullptr;
    int nu = 0, nw = 0, nx = 0;
    int64_t nv = 0;  // M2L (V list) pairs
    int* leaves = nullptr;
    int nleaves = 0;
    int* grp_tg = nullptr;          // boxes of levels >= 2 grouped by (level, octant)
    int* grp_ptr = nullptr;         // (maxlev + 1) * 8 + 1 offsets
    std::vector<int> grp_ptr_h;
    int a_exp_p = -1;               // order of the adaptive expansion arrays
    double *aM = nullptr, *aL = nullptr;
    float* aMf = nullptr;
    float* aMinv = nullptr;         // per box: factor of the F16 multipole split
    float* aLh = nullptr;           // harmonic-basis M2L output rows (FP32, free coefficients)
    size_t aLh_bytes = 0;
    float* aMc = nullptr;           // FP32 copy of the multipole rows for the leaves' M2P (FP32 paths)
    size_t aMc_bytes = 0;
};


namespace dafmm {
inline TreeView make_view(const dafmm_tree* t) {
    TreeView tv;
    tv.n = t->n;
    tv.depth = t->depth;
    tv.nleaf = t->nleaf;
    tv.x0 = t->dom[0]; tv.y0 = t->dom[1]; tv.z0 = t->dom[2]; tv.size = t->dom[3];
    tv.h_leaf = ldexp(t->dom[3], -t->depth);
    tv.inv_h_leaf = 1.0 / tv.h_leaf;
    tv.x = t->x; tv.y = t->y; tv.z = t->z; tv.q = t->q;
    tv.xq = t->xq;
    tv.perm = t->perm;
    tv.leaf_start = t->leaf_start;
    tv.locals_f32 = 0;
    return tv;
}
}  // namespace dafmm

struct dafmm_graph {
    dafmm_ctx* ctx = nullptr;
    dafmm_tree* tree = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
};

namespace dafmm {
// device allocation through a context (its budget or pool); used by other runtime units
int ctx_alloc(dafmm_ctx* c, void** p, size_t bytes, const char* what);
void ctx_free(dafmm_ctx* c, void* p, size_t bytes);
}  // namespace dafmm

// the uniform tree's build (if still asynchronous) ordered before work on stream s; the build's
// scratch is returned once the build has completed.  Returns a DAFMM code.
int tree_ready(dafmm_tree* t, cudaStream_t s);
