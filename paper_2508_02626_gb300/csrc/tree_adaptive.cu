// tree_adaptive.cu -- adaptive octree on the GPU (Sec. 3.5: a box with more than s particles
// is subdivided) and its interaction lists (Cheng, Greengard and Rokhlin 1999):
//   colleagues : same-level adjacent boxes, kept in a 27-slot table indexed by relative
//                position (slot 13 = the box itself), -1 where no box exists;
//   V (M2L)    : children of the parent's colleagues that are not adjacent -- looked up on
//                the fly from the colleague table by the evaluation kernels;
//   U (P2P)    : for a leaf, every leaf adjacent to it, and itself;
//   W (M2P)    : for a leaf b, descendants of its colleagues that are not adjacent to b but
//                whose parent is;
//   X (P2L)    : for a box b, the leaves c coarser than b that are adjacent to parent(b) and
//                not adjacent to b (exactly the boxes whose W list holds b).
// Particles are sorted by 63-bit Morton keys of their 21-bit integer coordinates, so every
// box is a contiguous particle range.  A forest holds several independent trees (one root
// box each, level 0): the particles are grouped by tree and sorted inside each tree, and no
// list ever crosses trees, since every relation is derived from the parent's colleagues.
#include <cuda_runtime.h>

#include "check.cuh"
#include "internal.h"
#include "tree_adaptive.h"
#include "tree_common.cuh"

namespace dafmm {

__device__ inline int quantize_a(double x, double x0, double scale) {
    double f = floor(__dmul_rn(__dsub_rn(x, x0), scale));
    const double top = (double)((1 << kQBits) - 1);
    if (!(f >= 0.0)) return 0;
    if (f > top) return (1 << kQBits) - 1;
    return (int)f;
}

__device__ inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// tree of particle i: the last r with offs[r] <= i
__device__ inline int tree_of(const int* offs, int nroots, int i) {
    int lo = 0, hi = nroots - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (offs[m] <= i) lo = m;
        else hi = m - 1;
    }
    return lo;
}

__global__ void k_morton_keys(const double* __restrict__ xyz, int64_t n, const int* __restrict__ offs, int nroots,
                              const double* __restrict__ rootdom, uint64_t* keys, int* vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = nroots > 1 ? tree_of(offs, nroots, (int)i) : 0;
    const double* d = rootdom + 4 * r;
    const double scale = ldexp(1.0, kQBits) / d[3];
    const uint32_t a = quantize_a(xyz[3 * i], d[0], scale);
    const uint32_t b = quantize_a(xyz[3 * i + 1], d[1], scale);
    const uint32_t c = quantize_a(xyz[3 * i + 2], d[2], scale);
    keys[i] = spread3(a) | (spread3(b) << 1) | (spread3(c) << 2);
    vals[i] = (int)i;
}

cudaError_t launch_morton_keys(const double* xyz, int64_t n, const int* offs, int nroots, const double* rootdom,
                               uint64_t* keys, int* vals, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_morton_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, n, offs, nroots, rootdom, keys, vals);
    return cudaGetLastError();
}

__global__ void k_tree_keys(const int* __restrict__ perm, int64_t n, const int* __restrict__ offs, int nroots,
                            uint64_t* tkeys, int* pos) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    tkeys[t] = (uint64_t)tree_of(offs, nroots, perm[t]);
    pos[t] = (int)t;
}

cudaError_t launch_tree_keys(const int* perm, int64_t n, const int* offs, int nroots, uint64_t* tkeys, int* pos,
                             cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_tree_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(perm, n, offs, nroots, tkeys, pos);
    return cudaGetLastError();
}

__global__ void k_apply_order(const int* __restrict__ pos, int64_t n, const int* __restrict__ perm_in,
                              const uint64_t* __restrict__ keys_in, int* perm_out, uint64_t* keys_out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int j = pos[t];
    perm_out[t] = perm_in[j];
    keys_out[t] = keys_in[j];
}

cudaError_t launch_apply_order(const int* pos, int64_t n, const int* perm_in, const uint64_t* keys_in, int* perm_out,
                               uint64_t* keys_out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_apply_order<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, perm_in, keys_in, perm_out, keys_out);
    return cudaGetLastError();
}

// order-preserving map of a double to an unsigned integer (for atomic min/max)
__device__ inline unsigned long long ordered_bits(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(256) k_bbox_roots(const double* __restrict__ xyz, const int* __restrict__ offs,
                                                    unsigned long long* bb) {
    const int r = blockIdx.x;
    const int b = offs[r], e = offs[r + 1];
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    for (int i = b + threadIdx.x; i < e; i += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const unsigned long long u = ordered_bits(xyz[3 * (size_t)i + d]);
            mn[d] = u < mn[d] ? u : mn[d];
            mx[d] = u > mx[d] ? u : mx[d];
        }
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[d], o);
            const unsigned long long c = __shfl_xor_sync(0xffffffffu, mx[d], o);
            mn[d] = a < mn[d] ? a : mn[d];
            mx[d] = c > mx[d] ? c : mx[d];
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bb[6 * r + d], mn[d]);
            atomicMax(&bb[6 * r + 3 + d], mx[d]);
        }
    }
}

__global__ void k_bbox_init(unsigned long long* bb, int nroots) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6 * nroots) bb[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

cudaError_t launch_bbox_roots(const double* xyz, const int* offs, int nroots, unsigned long long* bb, cudaStream_t s) {
    if (nroots == 0) return cudaSuccess;
    k_bbox_init<<<(6 * nroots + 255) / 256, 256, 0, s>>>(bb, nroots);
    k_bbox_roots<<<nroots, 256, 0, s>>>(xyz, offs, bb);
    return cudaGetLastError();
}

__global__ void k_box_geometry(const int* __restrict__ root, const int* __restrict__ level,
                               const int* __restrict__ ijk, const double* __restrict__ rootdom, int nbox,
                               double4* geom) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const double* d = rootdom + 4 * root[b];
    const double h = ldexp(d[3], -level[b]);
    geom[b] = make_double4(d[0] + ((double)ijk[3 * b] + 0.5) * h, d[1] + ((double)ijk[3 * b + 1] + 0.5) * h,
                           d[2] + ((double)ijk[3 * b + 2] + 0.5) * h, h);
}

cudaError_t launch_box_geometry(const int* root, const int* level, const int* ijk, const double* rootdom, int nbox,
                                double4* geom, cudaStream_t s) {
    if (nbox == 0) return cudaSuccess;
    k_box_geometry<<<(nbox + 255) / 256, 256, 0, s>>>(root, level, ijk, rootdom, nbox, geom);
    return cudaGetLastError();
}

// first sorted position in [b, e) whose level-(l+1) digit is >= c
__device__ inline int first_digit_ge(const uint64_t* keys, int b, int e, int shift, int c) {
    while (b < e) {
        const int m = (b + e) >> 1;
        if ((int)((keys[m] >> shift) & 7u) < c) b = m + 1;
        else e = m;
    }
    return b;
}

// per box of level l: number of non-empty children when it splits
__global__ void k_split_count(AdaptiveBuild ab, int lb, int le, int level, int max_leaf, int max_depth, int* nch) {
    const int b = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= le) return;
    const int pb = ab.pbeg[b], pe = ab.pend[b];
    int cnt = 0;
    if (pe - pb > max_leaf && level < max_depth) {
        const int shift = 3 * (kQBits - level - 1);
        int s = pb;
        for (int c = 0; c < 8; ++c) {
            const int e = first_digit_ge(ab.keys, s, pe, shift, c + 1);
            cnt += e > s;
            s = e;
        }
    }
    nch[b - lb] = cnt;
}

__global__ void k_split_fill(AdaptiveBuild ab, int lb, int le, int level, const int* offs, int first_new) {
    const int b = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= le) return;
    for (int c = 0; c < 8; ++c) ab.child[8 * b + c] = -1;
    const int k0 = offs[b - lb], k1 = offs[b - lb + 1];
    if (k0 == k1) return;
    const int pb = ab.pbeg[b], pe = ab.pend[b];
    const int shift = 3 * (kQBits - level - 1);
    int s = pb, k = first_new + k0;
    for (int c = 0; c < 8; ++c) {
        const int e = first_digit_ge(ab.keys, s, pe, shift, c + 1);
        if (e > s && DAFMM_IN(k, ab.cap, kChkSplitChild)) {
            ab.root[k] = ab.root[b];
            ab.level[k] = level + 1;
            ab.ijk[3 * k] = 2 * ab.ijk[3 * b] + (c & 1);
            ab.ijk[3 * k + 1] = 2 * ab.ijk[3 * b + 1] + ((c >> 1) & 1);
            ab.ijk[3 * k + 2] = 2 * ab.ijk[3 * b + 2] + ((c >> 2) & 1);
            ab.parent[k] = b;
            ab.pbeg[k] = s;
            ab.pend[k] = e;
            ab.child[8 * b + c] = k;
            ++k;
        }
        s = e;
    }
}

__global__ void k_leaf_children_init(int* child, int b0, int b1) {
    const int b = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (b < b1)
        for (int c = 0; c < 8; ++c) child[8 * b + c] = -1;
}

cudaError_t launch_split(AdaptiveBuild ab, int lb, int le, int level, int max_leaf, int max_depth, int* nch,
                         cudaStream_t s) {
    const int n = le - lb;
    if (n == 0) return cudaSuccess;
    k_split_count<<<(n + 127) / 128, 128, 0, s>>>(ab, lb, le, level, max_leaf, max_depth, nch);
    return cudaGetLastError();
}

cudaError_t launch_split_fill(AdaptiveBuild ab, int lb, int le, int level, const int* offs, int first_new,
                              cudaStream_t s) {
    const int n = le - lb;
    if (n == 0) return cudaSuccess;
    k_split_fill<<<(n + 127) / 128, 128, 0, s>>>(ab, lb, le, level, offs, first_new);
    return cudaGetLastError();
}

cudaError_t launch_children_init(int* child, int b0, int b1, cudaStream_t s) {
    if (b1 <= b0) return cudaSuccess;
    k_leaf_children_init<<<(b1 - b0 + 127) / 128, 128, 0, s>>>(child, b0, b1);
    return cudaGetLastError();
}

// exclusive scan of n ints by one block (n up to a few million; used at build time only); in
// and out are distinct, so the loads of a chunk need not wait for its stores
__global__ void __launch_bounds__(1024) k_scan_excl(const int* __restrict__ in, int* __restrict__ out, int n) {
    __shared__ int sums[1024];
    const int t = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int b = t * chunk, e = min(b + chunk, n);
    int s = 0;
#pragma unroll 8
    for (int i = b; i < e; ++i) s += in[i];
    sums[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int run = t ? sums[t - 1] : 0;
#pragma unroll 8
    for (int i = b; i < e; ++i) {
        const int v = in[i];
        out[i] = run;
        run += v;
    }
    if (t == 1023) out[n] = sums[1023];
}

cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t s) {
    k_scan_excl<<<1, 1024, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// ---- colleagues ---------------------------------------------------------------------------
__device__ inline bool same_level_adjacent(const int* ijk, int a, int b) {
    for (int d = 0; d < 3; ++d) {
        const int df = ijk[3 * a + d] - ijk[3 * b + d];
        if (df < -1 || df > 1) return false;
    }
    return true;
}

// closed cubes of two boxes (any levels) intersect
__device__ inline bool touch(const AdaptiveBuild& ab, int a, int b) {
    const int la = ab.level[a], lb = ab.level[b];
    const int L = la > lb ? la : lb;
    for (int d = 0; d < 3; ++d) {
        const int64_t alo = (int64_t)ab.ijk[3 * a + d] << (L - la), ahi = (int64_t)(ab.ijk[3 * a + d] + 1) << (L - la);
        const int64_t blo = (int64_t)ab.ijk[3 * b + d] << (L - lb), bhi = (int64_t)(ab.ijk[3 * b + d] + 1) << (L - lb);
        if (alo > bhi || blo > ahi) return false;
    }
    return true;
}

__global__ void k_colleagues(AdaptiveBuild ab, int lb, int le) {
    const int b = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= le) return;
    int* col = ab.colleague + 27 * b;
    for (int k = 0; k < 27; ++k) col[k] = -1;
    col[13] = b;
    const int P = ab.parent[b];
    if (P < 0) return;
    const int* pc = ab.colleague + 27 * P;
    for (int k = 0; k < 27; ++k) {
        const int Q = pc[k];
        if (Q < 0) continue;
        for (int c = 0; c < 8; ++c) {
            const int ch = ab.child[8 * Q + c];
            if (ch < 0 || ch == b) continue;
            if (!same_level_adjacent(ab.ijk, ch, b)) continue;
            const int dx = ab.ijk[3 * ch] - ab.ijk[3 * b], dy = ab.ijk[3 * ch + 1] - ab.ijk[3 * b + 1],
                      dz = ab.ijk[3 * ch + 2] - ab.ijk[3 * b + 2];
            col[(dx + 1) * 9 + (dy + 1) * 3 + (dz + 1)] = ch;
        }
    }
}

cudaError_t launch_colleagues(AdaptiveBuild ab, int lb, int le, cudaStream_t s) {
    if (le <= lb) return cudaSuccess;
    k_colleagues<<<(le - lb + 127) / 128, 128, 0, s>>>(ab, lb, le);
    return cudaGetLastError();
}

// ---- U, W (leaves) and X (all boxes) lists: count pass, then fill pass --------------------
constexpr int kStack = 256;

// U and W of leaf b: traverse the descendants of b's non-leaf colleagues; plus the same-level
// colleague leaves, plus coarser adjacent leaves (leaf colleagues of b's ancestors)
template <bool FILL>
__device__ void uw_lists(const AdaptiveBuild& ab, int b, int* nu, int* nw, int* ou, int* ow, int* err, int cap_u = 0,
                         int cap_w = 0) {
    int cu = 0, cw = 0;
    if (FILL && DAFMM_IN(cu, cap_u, kChkListFill)) ou[cu] = b;
    ++cu;
    const int* col = ab.colleague + 27 * b;
    int stack[kStack];
    for (int k = 0; k < 27; ++k) {
        const int c = col[k];
        if (c < 0 || c == b) continue;
        if (ab.child[8 * c] < 0 && ab.child[8 * c + 1] < 0 && ab.child[8 * c + 2] < 0 && ab.child[8 * c + 3] < 0 &&
            ab.child[8 * c + 4] < 0 && ab.child[8 * c + 5] < 0 && ab.child[8 * c + 6] < 0 && ab.child[8 * c + 7] < 0) {
            if (FILL && DAFMM_IN(cu, cap_u, kChkListFill)) ou[cu] = c;
            ++cu;
            continue;
        }
        int sp = 0;
        for (int j = 0; j < 8; ++j)
            if (ab.child[8 * c + j] >= 0) stack[sp++] = ab.child[8 * c + j];
        while (sp > 0) {
            const int x = stack[--sp];
            if (touch(ab, x, b)) {
                bool leaf = true;
                for (int j = 0; j < 8; ++j)
                    if (ab.child[8 * x + j] >= 0) {
                        leaf = false;
                        if (sp < kStack) stack[sp++] = ab.child[8 * x + j];
                        else atomicExch(err, 41);
                    }
                if (leaf) {
                    if (FILL && DAFMM_IN(cu, cap_u, kChkListFill)) ou[cu] = x;
                    ++cu;
                }
            } else {
                if (FILL && DAFMM_IN(cw, cap_w, kChkListFill)) ow[cw] = x;
                ++cw;
            }
        }
    }
    // coarser adjacent leaves
    for (int a = ab.parent[b]; a >= 0; a = ab.parent[a]) {
        const int* ac = ab.colleague + 27 * a;
        for (int k = 0; k < 27; ++k) {
            const int c = ac[k];
            if (c < 0 || c == a) continue;
            bool leaf = true;
            for (int j = 0; j < 8; ++j) leaf = leaf && ab.child[8 * c + j] < 0;
            if (leaf && touch(ab, c, b)) {
                if (FILL && DAFMM_IN(cu, cap_u, kChkListFill)) ou[cu] = c;
                ++cu;
            }
        }
    }
    *nu = cu;
    *nw = cw;
}

// X of box b: leaf colleagues c of b's ancestors (parent and up) adjacent to parent(b), not to b
template <bool FILL>
__device__ int x_list(const AdaptiveBuild& ab, int b, int* ox, int cap_x = 0) {
    const int P = ab.parent[b];
    if (P < 0) return 0;
    int cx = 0;
    for (int a = P; a >= 0; a = ab.parent[a]) {
        const int* ac = ab.colleague + 27 * a;
        for (int k = 0; k < 27; ++k) {
            const int c = ac[k];
            if (c < 0 || c == a) continue;
            bool leaf = true;
            for (int j = 0; j < 8; ++j) leaf = leaf && ab.child[8 * c + j] < 0;
            if (!leaf) continue;
            if (touch(ab, c, P) && !touch(ab, c, b)) {
                if (FILL && DAFMM_IN(cx, cap_x, kChkListFill)) ox[cx] = c;
                ++cx;
            }
        }
    }
    return cx;
}

// V of box b (counted only): children of the parent's colleagues that are not adjacent to b
__device__ int v_count(const AdaptiveBuild& ab, int b) {
    const int P = ab.parent[b];
    if (P < 0) return 0;
    int cv = 0;
    for (int k = 0; k < 27; ++k) {
        const int Q = ab.colleague[27 * P + k];
        if (Q < 0 || Q == P) continue;
        for (int c = 0; c < 8; ++c) {
            const int ch = ab.child[8 * Q + c];
            if (ch >= 0 && !same_level_adjacent(ab.ijk, ch, b)) ++cv;
        }
    }
    return cv;
}

__global__ void k_list_count(AdaptiveBuild ab, int nbox, int* cu, int* cw, int* cx, unsigned long long* nv,
                             int* err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    bool leaf = true;
    for (int j = 0; j < 8; ++j) leaf = leaf && ab.child[8 * b + j] < 0;
    int nu = 0, nw = 0;
    if (leaf) uw_lists<false>(ab, b, &nu, &nw, nullptr, nullptr, err);
    cu[b] = nu;
    cw[b] = nw;
    cx[b] = x_list<false>(ab, b, nullptr);
    const int v = v_count(ab, b);
    if (v) atomicAdd(nv, (unsigned long long)v);
}

__global__ void k_list_fill(AdaptiveBuild ab, int nbox, const int* pu, const int* pw, const int* px, int* iu, int* iw,
                            int* ix, int* err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    bool leaf = true;
    for (int j = 0; j < 8; ++j) leaf = leaf && ab.child[8 * b + j] < 0;
    int nu, nw;
    if (leaf) uw_lists<true>(ab, b, &nu, &nw, iu + pu[b], iw + pw[b], err, pu[b + 1] - pu[b], pw[b + 1] - pw[b]);
    x_list<true>(ab, b, ix + px[b], px[b + 1] - px[b]);
}

cudaError_t launch_list_count(AdaptiveBuild ab, int nbox, int* cu, int* cw, int* cx, unsigned long long* nv, int* err,
                              cudaStream_t s) {
    if (nbox == 0) return cudaSuccess;
    k_list_count<<<(nbox + 127) / 128, 128, 0, s>>>(ab, nbox, cu, cw, cx, nv, err);
    return cudaGetLastError();
}

cudaError_t launch_list_fill(AdaptiveBuild ab, int nbox, const int* pu, const int* pw, const int* px, int* iu, int* iw,
                             int* ix, int* err, cudaStream_t s) {
    if (nbox == 0) return cudaSuccess;
    k_list_fill<<<(nbox + 127) / 128, 128, 0, s>>>(ab, nbox, pu, pw, px, iu, iw, ix, err);
    return cudaGetLastError();
}

// ---- gather of the sorted particles: FP64 SoA and FP32 offsets in each particle's own leaf ----
__global__ void k_gather_adaptive(const double* __restrict__ xyz, const double* __restrict__ q,
                                  const int* __restrict__ perm, AdaptiveBuild ab, const int* __restrict__ leaves,
                                  int nleaves, const double4* __restrict__ geom, const int* __restrict__ xq0,
                                  double* x, double* y, double* z, double* qs, float4* xq, float4* xl, int64_t n,
                                  int64_t nrec) {
    const int li = blockIdx.x;
    if (li >= nleaves) return;
    const int b = leaves[li];
    if (!DAFMM_IN(b, ab.nbox, kChkBoxIndex) || !DAFMM_RANGE(ab.pbeg[b], ab.pend[b], n, kChkBoxRange)) return;
    const double4 g = geom[b];
    const double ih = 1.0 / g.w;
    const double cx = g.x, cy = g.y, cz = g.z;
    for (int t = ab.pbeg[b] + threadIdx.x; t < ab.pend[b]; t += blockDim.x) {
        const int i = perm[t];
        if (!DAFMM_IN(i, n, kChkPerm)) continue;
        const double px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2], pq = q[i];
        x[t] = px; y[t] = py; z[t] = pz; qs[t] = pq;
        const double ox = (px - cx) * ih, oy = (py - cy) * ih, oz = (pz - cz) * ih;
        const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
        const int r = xq0[b] + (t - ab.pbeg[b]);
        if (!DAFMM_IN(r, nrec, kChkRecord)) continue;
        xq_store(xq, r, hx, hy, hz, (float)pq);
        xq_store(xl, r, (float)(ox - (double)hx), (float)(oy - (double)hy), (float)(oz - (double)hz),
                 (float)(pq - (double)(float)pq));
    }
}

__global__ void k_leaf_pairs(const int* __restrict__ leaves, int nl, const int* __restrict__ pbeg,
                             const int* __restrict__ pend, int* cnt) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li < nl) {
        const int b = leaves[li];
        cnt[li] = (pend[b] - pbeg[b] + 1) >> 1;
    }
}

__global__ void k_leaf_xq0(const int* __restrict__ leaves, int nl, const int* __restrict__ off, int* xq0) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li < nl) xq0[leaves[li]] = 2 * off[li];
}

cudaError_t launch_leaf_records(const int* leaves, int nl, const int* pbeg, const int* pend, int* cnt, int* off,
                                int* xq0, cudaStream_t s) {
    if (nl == 0) return cudaSuccess;
    k_leaf_pairs<<<(nl + 255) / 256, 256, 0, s>>>(leaves, nl, pbeg, pend, cnt);
    cudaError_t e = launch_scan(cnt, off, nl, s);
    if (e != cudaSuccess) return e;
    k_leaf_xq0<<<(nl + 255) / 256, 256, 0, s>>>(leaves, nl, off, xq0);
    return cudaGetLastError();
}

cudaError_t launch_gather_adaptive(const double* xyz, const double* q, const int* perm, AdaptiveBuild ab,
                                   const int* leaves, int nleaves, const double4* geom, const int* xq0, double* x,
                                   double* y, double* z, double* qs, float4* xq, size_t xq_n4, int64_t n, cudaStream_t s) {
    // the zero fill supplies the padding record of leaves with an odd particle count (both
    // halves: the records and their remainders)
    cudaError_t e = cudaMemsetAsync(xq, 0, 2 * xq_n4 * sizeof(float4), s);
    if (e != cudaSuccess || nleaves == 0) return e;
    k_gather_adaptive<<<nleaves, 128, 0, s>>>(xyz, q, perm, ab, leaves, nleaves, geom, xq0, x, y, z, qs, xq,
                                              xq + xq_n4, n, (int64_t)xq_n4);
    return cudaGetLastError();
}

// ---- leaves and M2L target groups --------------------------------------------------------------
__global__ void k_leaf_flags(const int* __restrict__ child, int nbox, int* flags) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    bool leaf = true;
    for (int j = 0; j < 8; ++j) leaf = leaf && child[8 * b + j] < 0;
    flags[b] = leaf ? 1 : 0;
}

__global__ void k_scatter_flagged(const int* __restrict__ flags, const int* __restrict__ offs, int nbox, int* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox && flags[b]) out[offs[b]] = b;
}

// group key (level, octant) of the boxes of levels >= 2; other boxes sort last
__global__ void k_group_keys(const int* __restrict__ level, const int* __restrict__ ijk, int nbox, uint64_t* keys,
                             int* vals) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int l = level[b];
    const int oct = (ijk[3 * b] & 1) | ((ijk[3 * b + 1] & 1) << 1) | ((ijk[3 * b + 2] & 1) << 2);
    keys[b] = l >= 2 ? (uint64_t)(l * 8 + oct) : 0xffu;
    vals[b] = b;
}

__global__ void k_group_ptr(const uint64_t* __restrict__ keys, int n, int ngroups, int* ptr) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > ngroups) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (keys[m] < (uint64_t)g) lo = m + 1;
        else hi = m;
    }
    ptr[g] = lo;
}

cudaError_t launch_leaf_flags(const int* child, int nbox, int* flags, cudaStream_t s) {
    if (nbox == 0) return cudaSuccess;
    k_leaf_flags<<<(nbox + 255) / 256, 256, 0, s>>>(child, nbox, flags);
    return cudaGetLastError();
}

cudaError_t launch_scatter_flagged(const int* flags, const int* offs, int nbox, int* out, cudaStream_t s) {
    if (nbox == 0) return cudaSuccess;
    k_scatter_flagged<<<(nbox + 255) / 256, 256, 0, s>>>(flags, offs, nbox, out);
    return cudaGetLastError();
}

cudaError_t launch_group_keys(const int* level, const int* ijk, int nbox, uint64_t* keys, int* vals, cudaStream_t s) {
    if (nbox == 0) return cudaSuccess;
    k_group_keys<<<(nbox + 255) / 256, 256, 0, s>>>(level, ijk, nbox, keys, vals);
    return cudaGetLastError();
}

cudaError_t launch_group_ptr(const uint64_t* keys, int n, int ngroups, int* ptr, cudaStream_t s) {
    k_group_ptr<<<(ngroups + 1 + 255) / 256, 256, 0, s>>>(keys, n, ngroups, ptr);
    return cudaGetLastError();
}

}  // namespace dafmm
