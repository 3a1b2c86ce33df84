// Host-side check of the pair-interleaved FP32 particle records of tree_common.cuh (xq_base,
// xq_records, xq_store, xq_load), compiled by tests/test_xq_layout.py with g++; no GPU.
// Returns 0 when every property holds, else the number of the first failed property.
#include <cstring>
#include <random>
#include <vector>

#include "tree_common.cuh"

using namespace dafmm;

#ifdef PLANT_ODD_BASE
// a planted mistake: leaves placed without the rounding to an even record
#define xq_base(p, g) ((p) + (g))
#endif

namespace {

// one partition of n particles into g leaves (counts cnt, sorted order): the leaves' record
// ranges, pad included, must start even, stay inside xq_records(n, g), and be disjoint; no
// pair of records may span two leaves
int check_partition(const std::vector<int>& cnt) {
    const int g = (int)cnt.size();
    int64_t n = 0;
    for (int c : cnt) n += c;
    const size_t total = xq_records(n, g);
    if (total % 2) return 1;  // whole pairs
    std::vector<int> owner(total, -1);
    int start = 0;  // leaf_start[l]
    for (int l = 0; l < g; ++l) {
        const int b = xq_base(start, l);
        if (b % 2 || b < 0) return 2;
        const int len = cnt[l] + (cnt[l] & 1);  // the zero record completes an odd leaf
        if ((size_t)b + len > total) return 3;
        for (int r = b; r < b + len; ++r) {
            if (owner[r] != -1) return 4;
            owner[r] = l;
        }
        start += cnt[l];
    }
    for (size_t p = 0; p < total / 2; ++p)
        if (owner[2 * p] != owner[2 * p + 1] && owner[2 * p] != -1 && owner[2 * p + 1] != -1) return 5;
    return 0;
}

}  // namespace

extern "C" int xq_layout_check(unsigned seed) {
    std::mt19937 rng(seed);
    // fixed cases: no particles, one leaf, empty leaves between odd ones
    const std::vector<std::vector<int>> fixed = {{}, {0}, {1}, {2}, {3}, {0, 0, 0}, {1, 0, 1},
                                                 {3, 0, 0, 5, 1}, {2, 2, 2}, {1, 1, 1, 1, 1}};
    for (const auto& c : fixed)
        if (int e = check_partition(c)) return 10 + e;
    std::uniform_int_distribution<int> G(1, 300), C(0, 70), Z(0, 3);
    for (int trial = 0; trial < 400; ++trial) {
        std::vector<int> cnt(G(rng));
        for (int& c : cnt) c = Z(rng) == 0 ? 0 : C(rng);
        if (int e = check_partition(cnt)) return 20 + e;
    }
    // the interleave: records 2p and 2p + 1 as (x, x', y, y') (z, z', q, q'), and the round trip
    const int R = 37;
    std::vector<float4> xq((R + 1) / 2 * 2);
    std::memset(xq.data(), 0, xq.size() * sizeof(float4));
    for (int r = 0; r < R; ++r) xq_store(xq.data(), r, 1.f + r, 100.f + r, 200.f + r, 300.f + r);
    for (int r = 0; r < R; ++r) {
        const float4 v = xq_load(xq.data(), r);
        if (v.x != 1.f + r || v.y != 100.f + r || v.z != 200.f + r || v.w != 300.f + r) return 30;
        const float4 A = xq[2 * (r / 2)], B = xq[2 * (r / 2) + 1];
        const float* a = &A.x;
        const float* b = &B.x;
        const int h = r % 2;
        if (a[h] != 1.f + r || a[2 + h] != 100.f + r || b[h] != 200.f + r || b[2 + h] != 300.f + r) return 31;
    }
    return 0;
}

// the octant-major box index of level l: a bijection of the 8^l boxes onto [0, 8^l), inverted
// by octmajor_decode, with the 8 children of a parent at one offset of the 8 octant slabs
// (child octant o of parent (I, J, K) at o * 8^(l-1) + the parent's index at level l - 1)
extern "C" int octmajor_check(int l) {
    const int s = 1 << l, nbox = s * s * s;
    std::vector<int> seen(nbox, 0);
    for (int k = 0; k < s; ++k)
        for (int j = 0; j < s; ++j)
            for (int i = 0; i < s; ++i) {
                const int idx = octmajor_index(l, i, j, k);
                if (idx < 0 || idx >= nbox || seen[idx]) return 1;
                seen[idx] = 1;
                int a, b, c;
                octmajor_decode(l, idx, a, b, c);
                if (a != i || b != j || c != k) return 2;
                if (l >= 1) {
                    const int P3 = nbox / 8;
                    const int oct = (i & 1) | (j & 1) << 1 | (k & 1) << 2;
                    // the parent's position in its own level, as a plain row-major grid of P^3
                    const int P = s / 2, par = ((k >> 1) * P + (j >> 1)) * P + (i >> 1);
                    if (idx != oct * P3 + par) return 3;
                }
            }
    return 0;
}
