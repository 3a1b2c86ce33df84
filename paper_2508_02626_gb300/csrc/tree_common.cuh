// tree_common.cuh -- box indexing shared by the kernels.
//
// Boxes of level l of a uniform tree are stored "octant-major": the box with integer
// coordinates (i, j, k) sits at
//     index = oct * P^3 + ((k >> 1) * P + (j >> 1)) * P + (i >> 1),   P = 2^(l-1),
//     oct   = (i & 1) | (j & 1) << 1 | (k & 1) << 2,
// i.e. one dense grid of parents per child octant.  The eight children of a parent are
// then at the same offset of the eight octant slabs (M2M, L2L), and all targets of one
// octant share the same 189 M2L displacements (Sec. 3.4).
#pragma once

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

}  // namespace dafmm
