// tree_build.cu -- octree construction on the GPU: bounding cube, box keys, a stable LSD
// radix sort of (key, particle) pairs, and the gather of the sorted particle arrays.
//
// Box membership follows one rule on every path (host oracle included):
//     k = clamp(floor((x - x0) * (2^21 / size)), 0, 2^21 - 1)   per axis,
// computed with explicitly rounded double operations so that no contraction changes it.
#include <cuda_runtime.h>

#include "check.cuh"
#include "internal.h"
#include "tree_common.cuh"

namespace dafmm {

// ---- bounding box -------------------------------------------------------------------------
// order-preserving map of doubles onto unsigned 64-bit integers (for atomic min/max)
__device__ inline unsigned long long ord_encode(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_bbox(const double* __restrict__ xyz, int64_t n, unsigned long long* out6) {
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; ++d) {
            unsigned long long e = ord_encode(xyz[3 * i + d]);
            lo[d] = e < lo[d] ? e : lo[d];
            hi[d] = e > hi[d] ? e : hi[d];
        }
    }
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[d], o);
            unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[d], o);
            lo[d] = a < lo[d] ? a : lo[d];
            hi[d] = b > hi[d] ? b : hi[d];
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&out6[d], lo[d]);
            atomicMax(&out6[3 + d], hi[d]);
        }
    }
}

__global__ void k_bbox_init(unsigned long long* out6) {
    if (threadIdx.x < 3) out6[threadIdx.x] = ~0ull;
    else if (threadIdx.x < 6) out6[threadIdx.x] = 0ull;
}

cudaError_t launch_bbox(const double* xyz, int64_t n, double* out6, cudaStream_t s) {
    unsigned long long* o = reinterpret_cast<unsigned long long*>(out6);
    k_bbox_init<<<1, 32, 0, s>>>(o);
    if (n > 0) {
        int blocks = (int)((n + 255) / 256);
        if (blocks > 152 * 8) blocks = 152 * 8;
        k_bbox<<<blocks, 256, 0, s>>>(xyz, n, o);
    }
    return cudaGetLastError();
}

// ---- keys ---------------------------------------------------------------------------------
__device__ inline int quantize(double x, double x0, double scale) {
    double f = floor(__dmul_rn(__dsub_rn(x, x0), scale));
    const double top = (double)((1 << kQBits) - 1);
    if (!(f >= 0.0)) return 0;  // also maps NaN to 0
    if (f > top) return (1 << kQBits) - 1;
    return (int)f;
}

__global__ void k_uniform_keys(const double* __restrict__ xyz, int64_t n, double x0, double y0,
                               double z0, double scale, int depth, uint64_t* keys, int* vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sh = kQBits - depth;
    int a = quantize(xyz[3 * i], x0, scale) >> sh;
    int b = quantize(xyz[3 * i + 1], y0, scale) >> sh;
    int c = quantize(xyz[3 * i + 2], z0, scale) >> sh;
    keys[i] = (uint64_t)octmajor_index(depth, a, b, c);
    vals[i] = (int)i;
}

cudaError_t launch_uniform_keys(const double* xyz, int64_t n, double x0, double y0, double z0,
                                double scale, int depth, uint64_t* keys, int* vals, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_uniform_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, n, x0, y0, z0, scale, depth, keys, vals);
    return cudaGetLastError();
}

// ---- stable LSD radix sort, 8-bit digits --------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                        int shift, unsigned* hist, int nb) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of `total` counters by one block of 1024 threads.  Each thread owns a chunk of
// a multiple of 4 counters (16-byte aligned: hist is) and reads it with 16-byte loads, eight in
// flight, so each pass over the counters costs a few memory round trips rather than one per
// counter.
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned* __restrict__ hist, int total) {
    __shared__ unsigned sums[1024];
    const int t = threadIdx.x;
    const int chunk = ((total + 1023) / 1024 + 3) & ~3;
    const int b = min(t * chunk, total), e = min(b + chunk, total);
    const int ev = b + (e - b) / 4 * 4;  // end of the whole 4-counter groups
    unsigned s = 0;
#pragma unroll 8
    for (int i = b; i < ev; i += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(hist + i);
        s += v.x + v.y + v.z + v.w;
    }
    for (int i = ev; i < e; ++i) s += hist[i];
    sums[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        unsigned v = t >= off ? sums[t - off] : 0u;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    unsigned run = t ? sums[t - 1] : 0u;
    // in place: a batch of 8 groups is read before any of it is written
    for (int i0 = b; i0 < ev; i0 += 32) {
        uint4 v[8];
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (i0 + 4 * g < ev) v[g] = *reinterpret_cast<const uint4*>(hist + i0 + 4 * g);
#pragma unroll
        for (int g = 0; g < 8; ++g)
            if (i0 + 4 * g < ev) {
                const uint4 o = make_uint4(run, run + v[g].x, run + v[g].x + v[g].y, run + v[g].x + v[g].y + v[g].z);
                run += v[g].x + v[g].y + v[g].z + v[g].w;
                *reinterpret_cast<uint4*>(hist + i0 + 4 * g) = o;
            }
    }
    for (int i = ev; i < e; ++i) {
        const unsigned v = hist[i];
        hist[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                           const int* __restrict__ vin,
                                                           uint64_t* __restrict__ kout,
                                                           int* __restrict__ vout, int64_t n, int shift,
                                                           const unsigned* __restrict__ offs, int nb) {
    __shared__ unsigned base[256];
    __shared__ unsigned wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    base[tid] = offs[tid * nb + blockIdx.x];
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int ww = 0; ww < RS_THREADS / 32; ++ww) wcnt[ww][tid] = 0u;  // own column only
        __syncthreads();
        const int64_t i = tile + r * RS_THREADS + tid;
        const bool valid = i < n;
        const uint64_t k = valid ? kin[i] : 0ull;
        const int v = valid ? vin[i] : 0;
        const unsigned d = valid ? ((unsigned)(k >> shift) & 255u) : 256u;
        const unsigned mask = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(mask & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[w][d] = __popc(mask);
        __syncthreads();
        if (valid) {
            unsigned pos = base[d] + rank;
            for (int ww = 0; ww < w; ++ww) pos += wcnt[ww][d];
            if (DAFMM_IN(pos, n, kChkSortScatter)) {
                kout[pos] = k;
                vout[pos] = v;
            }
        }
        __syncthreads();
        unsigned tot = 0;
        for (int ww = 0; ww < RS_THREADS / 32; ++ww) tot += wcnt[ww][tid];
        base[tid] += tot;
    }
}

static int rs_blocks(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

size_t radix_sort_temp_bytes(int64_t n) {
    size_t nb = (size_t)(rs_blocks(n) > 0 ? rs_blocks(n) : 1);
    return (size_t)n * (sizeof(uint64_t) + sizeof(int)) + 256 * nb * sizeof(unsigned) + 256;
}

cudaError_t radix_sort_pairs(uint64_t* keys, int* vals, int64_t n, int bits, void* temp, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int nb = rs_blocks(n);
    if ((int64_t)nb * 256 > (int64_t)1 << 30) return cudaErrorInvalidValue;
    char* t = static_cast<char*>(temp);
    uint64_t* k2 = reinterpret_cast<uint64_t*>(t);
    int* v2 = reinterpret_cast<int*>(t + (size_t)n * sizeof(uint64_t));
    size_t off = (size_t)n * (sizeof(uint64_t) + sizeof(int));
    off = (off + 255) / 256 * 256;
    unsigned* hist = reinterpret_cast<unsigned*>(t + off);
    uint64_t *ka = keys, *kb = k2;
    int *va = vals, *vb = v2;
    const int npass = (bits + 7) / 8;
    for (int pass = 0; pass < npass; ++pass) {
        const int shift = 8 * pass;
        k_rs_hist<<<nb, RS_THREADS, 0, s>>>(ka, n, shift, hist, nb);
        k_rs_scan<<<1, 1024, 0, s>>>(hist, 256 * nb);
        k_rs_scatter<<<nb, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
        uint64_t* tk = ka; ka = kb; kb = tk;
        int* tv = va; va = vb; vb = tv;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ka != keys) {
        e = cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals, va, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s);
    }
    return e;
}

// ---- gather -----------------------------------------------------------------------------
__global__ void k_gather_uniform(const double* __restrict__ xyz, const double* __restrict__ q,
                                 const int* __restrict__ perm, int64_t n,
                                 const uint64_t* __restrict__ keys, TreeView tv, double* x, double* y,
                                 double* z, double* qs, float4* xq, float4* xl) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = perm[t];
    if (!DAFMM_IN(i, n, kChkPerm) || !DAFMM_IN(keys[t], tv.nleaf, kChkLeafKey)) return;
    const double px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2], pq = q[i];
    x[t] = px; y[t] = py; z[t] = pz; qs[t] = pq;
    int a, b, c;
    octmajor_decode(tv.depth, (int)keys[t], a, b, c);
    const double cx = tv.x0 + ((double)a + 0.5) * tv.h_leaf;
    const double cy = tv.y0 + ((double)b + 0.5) * tv.h_leaf;
    const double cz = tv.z0 + ((double)c + 0.5) * tv.h_leaf;
    const int leaf = (int)keys[t], p0 = tv.leaf_start[leaf];
    const double ox = (px - cx) * tv.inv_h_leaf, oy = (py - cy) * tv.inv_h_leaf, oz = (pz - cz) * tv.inv_h_leaf;
    const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
    const int r = xq_base(p0, leaf) + (int)(t - p0);
    if (!DAFMM_IN(r, xq_records(n, tv.nleaf), kChkRecord)) return;
    xq_store(xq, r, hx, hy, hz, (float)pq);
    xq_store(xl, r, (float)(ox - (double)hx), (float)(oy - (double)hy), (float)(oz - (double)hz),
             (float)(pq - (double)(float)pq));
}

__global__ void k_leaf_ranges(const uint64_t* __restrict__ keys, int64_t n, int nleaf, int* leaf_start) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nleaf) return;
    // first sorted position whose key is >= b
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < (uint64_t)b) lo = mid + 1;
        else hi = mid;
    }
    leaf_start[b] = (int)lo;
}

cudaError_t launch_gather_uniform(const double* xyz, const double* q, const int* perm, int64_t n,
                                  const uint64_t* sorted_keys, TreeView tv, double* x, double* y,
                                  double* z, double* qs, float4* xq, int* leaf_start, cudaStream_t s) {
    // leaf ranges first: the gather places each leaf's FP32 records from its first position;
    // the zero fill supplies the padding record of odd leaves
    k_leaf_ranges<<<(tv.nleaf + 1 + 255) / 256, 256, 0, s>>>(sorted_keys, n, tv.nleaf, leaf_start);
    // (both halves: the records and their remainders)
    const size_t n4 = xq_records(n, tv.nleaf);
    cudaError_t e = cudaMemsetAsync(xq, 0, 2 * n4 * sizeof(float4), s);
    if (e != cudaSuccess) return e;
    tv.leaf_start = leaf_start;
    if (n > 0)
        k_gather_uniform<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, q, perm, n, sorted_keys, tv, x,
                                                                     y, z, qs, xq, xq + n4);
    return cudaGetLastError();
}

__global__ void k_scatter_out(const double* __restrict__ ps, const double* __restrict__ fs,
                              const int* __restrict__ perm, int64_t n, double* phi, double* field) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = perm[t];
    if (!DAFMM_IN(i, n, kChkPerm)) return;
    if (phi) phi[i] = ps[t];
    if (field)
        for (int d = 0; d < 3; ++d) field[3 * i + d] = fs[3 * t + d];
}

cudaError_t launch_scatter_outputs(const double* phi_sorted, const double* field_sorted, const int* perm,
                                   int64_t n, double* phi, double* field, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_scatter_out<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi_sorted, field_sorted, perm, n, phi, field);
    return cudaGetLastError();
}

}  // namespace dafmm
