// tree_common.cuh -- box indexing shared by the kernels.
//
// Boxes of level l of a uniform tree are stored "octant-major": the box with integer
// coordinates (i, j, k) sits at
//     index = oct * P^3 + ((k >> 1) * P + (j >> 1)) * P + (i >> 1),   P = 2^(l-1),
//     oct   = (i & 1) | (j & 1) << 1 | (k & 1) << 2,
// i.e. one dense grid of parents per child octant.  The eight children of a parent are
// then at the same offset of the eight octant slabs (M2M, L2L), and all targets of one
// octant share the same 189 M2L displacements (Sec. 3.4).
//
// The FP32 particle records of the near field (leaf-frame offsets and charge) are stored
// pair-interleaved: pair p = records 2p and 2p + 1 occupies two float4s,
//     (x_2p, x_2p+1, y_2p, y_2p+1)  and  (z_2p, z_2p+1, q_2p, q_2p+1),
// so that one 16-byte load yields the x and the y of both particles as aligned float2 pairs
// for the packed FP32x2 instructions of the pairwise sum.  The records of every leaf start at
// an even record, and a leaf with an odd particle count ends in one zero record (q = 0 at the
// leaf centre, which adds exactly nothing), so the pairs of a leaf never depend on where its
// particles sit in the sorted order: a member of a forest sums its near field exactly as the
// same tree built alone.  A uniform tree, whose leaf index grows with the sorted position,
// places leaf l at xq_base(leaf_start[l], l); an adaptive tree keeps a table of first records
// per leaf box.  n particles in g leaves take at most xq_records(n, g) records = float4s.
//
// The record array holds two such halves of xq_records(n, g) float4s each: the first holds
// the offsets rounded to FP32 (hi) and the charge rounded to FP32, the second, at the same
// record index, the FP32 remainders lo = fl(v - hi) of the three offsets and of the charge.  hi + lo carries
// the offset to about 2^-48 leaf widths, so the near field can form the difference of two
// close particles from both parts with a relative error of a few FP32 roundings instead of
// the 2^-25 leaf widths of the rounded offsets alone (which dominated the field's error
// through the closest pairs).
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <vector_functions.h>
#include <vector_types.h>

namespace dafmm {

__host__ __device__ inline int octmajor_index(int l, int i, int j, int k) {
    if (l == 0) return 0;
    const int P = 1 << (l - 1);
    const int oct = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    return oct * P * P * P + (((k >> 1) * P + (j >> 1)) * P + (i >> 1));
}

__host__ __device__ inline void octmajor_decode(int l, int idx, int& i, int& j, int& k) {
    if (l == 0) {
        i = j = k = 0;
        return;
    }
    const int P = 1 << (l - 1);
    const int P3 = P * P * P;
    const int oct = idx / P3;
    const int lin = idx - oct * P3;
    const int px = lin % P, py = (lin / P) % P, pz = lin / (P * P);
    i = 2 * px + (oct & 1);
    j = 2 * py + ((oct >> 1) & 1);
    k = 2 * pz + ((oct >> 2) & 1);
}

__host__ __device__ inline int xq_base(int p, int g) { return (p + g + 1) & ~1; }
__host__ __device__ inline size_t xq_records(int64_t n, int64_t groups) { return (size_t)(n + groups + 3) & ~size_t(1); }

__device__ __forceinline__ void xq_store(float4* xq, int r, float x, float y, float z, float q) {
    float* f = reinterpret_cast<float*>(xq) + 8 * (r >> 1) + (r & 1);
    f[0] = x;
    f[2] = y;
    f[4] = z;
    f[6] = q;
}

// record r as (x, y, z, q)
__device__ __forceinline__ float4 xq_load(const float4* xq, int r) {
    const float* f = reinterpret_cast<const float*>(xq) + 8 * (r >> 1) + (r & 1);
    return make_float4(f[0], f[2], f[4], f[6]);
}

}  // namespace dafmm
