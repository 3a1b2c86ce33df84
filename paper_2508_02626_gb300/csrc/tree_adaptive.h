// tree_adaptive.h -- device arrays of an adaptive octree and the build launchers
// (tree_adaptive.cu).  Boxes are numbered breadth-first, so each level is a contiguous
// index range; every box is a contiguous range of the Morton-sorted particles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dafmm {

constexpr int kMaxAdaptiveDepth = 20;

struct AdaptiveBuild {
    const uint64_t* keys;  // sorted Morton keys of the particles
    int* root;             // per box: the tree (root box) it belongs to
    int* level;            // per box
    int* ijk;              // per box, 3 integer coordinates at its level
    int* parent;           // -1 for the root
    int* child;            // per box, 8 slots (octant c = x | y<<1 | z<<2), -1 when absent
    int* pbeg;             // particle range [pbeg, pend) in sorted order
    int* pend;
    int* colleague;        // per box, 27 slots by relative position, slot 13 = the box
#if defined(DAFMM_CHECK)
    int cap;               // checked builds: boxes the arrays hold, and (once the levels are
    int nbox;              // built) the boxes of the tree
#endif
};

// what the evaluation kernels read (const view)
struct AdaptiveView {
    int nbox;
    const int* level;
    const int* ijk;
    const int* parent;
    const int* child;
    const int* pbeg;
    const int* pend;
    const int* colleague;
    const int* u_ptr;      // CSR per box (empty for non-leaves)
    const int* u_idx;
    const int* w_ptr;
    const int* w_idx;
    const int* x_ptr;      // CSR per box
    const int* x_idx;
    const double4* geom;   // per box: centre x, y, z and width h
    const double *x, *y, *z, *q;  // sorted particles
    const float4* xq;             // offsets in the particle's own leaf, in leaf widths, and q (FP32,
                                  // pair-interleaved records, those of leaf box b from xq0[b])
    const float4* xl;             // the FP32 remainders of those offsets, same records
    const int* xq0;               // per leaf box: its first record (even)
    const int* perm;
#if defined(DAFMM_CHECK)
    int64_t n, nrec;              // checked builds: particles, FP32 records (one half of xq),
    int nu, nw, nx;               // U / W / X list entries (the bounds of the index checks)
#endif
};

// Morton keys of particles grouped by tree: particles [offs[r], offs[r+1]) belong to tree r,
// whose root cube is rootdom[4r .. 4r+3] = {x0, y0, z0, size}
cudaError_t launch_morton_keys(const double* xyz, int64_t n, const int* offs, int nroots, const double* rootdom,
                               uint64_t* keys, int* vals, cudaStream_t s);
// after the Morton sort: regroup by tree, keeping the Morton order inside each tree (stable)
cudaError_t launch_tree_keys(const int* perm, int64_t n, const int* offs, int nroots, uint64_t* tkeys, int* pos,
                             cudaStream_t s);
cudaError_t launch_apply_order(const int* pos, int64_t n, const int* perm_in, const uint64_t* keys_in, int* perm_out,
                               uint64_t* keys_out, cudaStream_t s);
// per-tree bounding boxes as ordered-integer min/max (6 per tree), one CTA per tree
cudaError_t launch_bbox_roots(const double* xyz, const int* offs, int nroots, unsigned long long* bb, cudaStream_t s);
cudaError_t launch_box_geometry(const int* root, const int* level, const int* ijk, const double* rootdom, int nbox,
                                double4* geom, cudaStream_t s);
cudaError_t launch_split(AdaptiveBuild ab, int lb, int le, int level, int max_leaf, int max_depth, int* nch,
                         cudaStream_t s);
cudaError_t launch_split_fill(AdaptiveBuild ab, int lb, int le, int level, const int* offs, int first_new,
                              cudaStream_t s);
cudaError_t launch_children_init(int* child, int b0, int b1, cudaStream_t s);
cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t s);  // out[n] = total
cudaError_t launch_colleagues(AdaptiveBuild ab, int lb, int le, cudaStream_t s);
cudaError_t launch_list_count(AdaptiveBuild ab, int nbox, int* cu, int* cw, int* cx, unsigned long long* nv, int* err,
                              cudaStream_t s);
cudaError_t launch_list_fill(AdaptiveBuild ab, int nbox, const int* pu, const int* pw, const int* px, int* iu, int* iw,
                             int* ix, int* err, cudaStream_t s);
// first FP32 record of every leaf box (xq0[b], even): the leaves of the list take consecutive
// record ranges of 2 ceil(n / 2) records; cnt and off are scratch of nl and nl + 1 ints
cudaError_t launch_leaf_records(const int* leaves, int nl, const int* pbeg, const int* pend, int* cnt, int* off,
                                int* xq0, cudaStream_t s);
cudaError_t launch_gather_adaptive(const double* xyz, const double* q, const int* perm, AdaptiveBuild ab,
                                   const int* leaves, int nleaves, const double4* geom, const int* xq0, double* x,
                                   double* y, double* z, double* qs, float4* xq, size_t xq_n4, int64_t n, cudaStream_t s);

cudaError_t launch_leaf_flags(const int* child, int nbox, int* flags, cudaStream_t s);
cudaError_t launch_scatter_flagged(const int* flags, const int* offs, int nbox, int* out, cudaStream_t s);
cudaError_t launch_group_keys(const int* level, const int* ijk, int nbox, uint64_t* keys, int* vals, cudaStream_t s);
cudaError_t launch_group_ptr(const uint64_t* keys, int n, int ngroups, int* ptr, cudaStream_t s);

}  // namespace dafmm
