// fmm_order.cuh -- the FMM kernels of one expansion order (DAFMM_P), instantiated by fmm_p*.cu.
//
// Every expansion is stored in box-scaled variables (a box of width h becomes width 1):
//   multipole M~_a = M_a / h^|a|,  local L~_b = L_b h^|b|,
// so P2M/L2P/M2P use offsets divided by h, M2M and L2L are level-independent tables, and
// M2L is L~ = (1/h) K^_v M~ with K^_v depending only on the integer box displacement v.
//
// Kernels (paper operator -> kernel):
//   P2M  (Eq. 2)  k_p2m       one warp per leaf; each lane runs the generated straight-line
//                             P2M of one particle, a padded shared-memory transpose sums the
//                             32 lanes per coefficient
//   M2M  (Eq. 4)  k_m2m       32 parents per block; the 8 octant maps are one table with sign
//                             flips (Sec. 3.3)
//   M2L  (Eq. 5)  k_kgen      K^_v for all 316 displacements, FP64 numerical DA products of the
//                             generated transfer map (one block per v)
//                 k_m2l       L~_t = (1/h) sum_v K^_v M~_{t-v} over the 189 displacements of
//                             the target's octant (SIMT, FP64 or FP32)
//   L2L  (Eq. 7)  k_l2l       32 parents per block, 8 child tables by sign flips
//   L2P + P2P     k_leaf      one warp per target leaf: pairwise sum over the 27 neighbour
//                             leaves and the generated L2P of the leaf's local expansion
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "da_common.cuh"
#include "check.cuh"
#include "ff.cuh"
#include "internal.h"
#include "tree_adaptive.h"
#include "tree_common.cuh"

#define DAFMM_CAT_(a, b) a##b
#define DAFMM_CAT(a, b) DAFMM_CAT_(a, b)
#define DAFMM_STR_(a) #a
#define DAFMM_STR(a) DAFMM_STR_(a)
#include DAFMM_STR(DAFMM_CAT(generated/da_ops_p, DAFMM_P).cuh)
#include DAFMM_STR(DAFMM_CAT(generated/da_tables_p, DAFMM_P).h)

#define GEN(name) DAFMM_CAT(name, DAFMM_CAT(_o, DAFMM_P))
#define GENT(name, suffix) DAFMM_CAT(GEN(name), suffix)

namespace dafmm {
namespace DAFMM_CAT(ord_, DAFMM_P) {

constexpr int P = DAFMM_P;
constexpr int NC = ncoef_of(P);
constexpr int NCP = ncp_of(P);

template <class T>
struct SmemSink {
    T* base;
    int lane;
    __device__ __forceinline__ void operator()(int k, T v) const { base[k * 33 + lane] = v; }
};

// Sums one coefficient per lane over the warp's 32 particles while the generated code emits
// the coefficients in increasing order: every 32 coefficients the [32][33] staging block is
// reduced row by row (lane j takes coefficient 32 c + j), so the staging needs 32 x 33
// values per warp instead of ncoef x 33.  The generated code passes k as a constant, so the
// flush tests fold away.
// NO: the number of coefficients the generated code emits (NC; the harmonic P2M: (p + 1)^2).
template <class T, int NJ, int NO = NC>
struct ChunkSink {
    T* buf;       // [32][33] per warp
    int lane;
    T (&acc)[NJ];  // acc[c] += coefficient 32 c + lane
    __device__ __forceinline__ void operator()(int k, T v) const {
        buf[(k & 31) * 33 + lane] = v;
        if ((k & 31) == 31 || k == NO - 1) {
            __syncwarp();
            if (lane <= (k & 31)) {
                T s = T(0);
#pragma unroll 8
                for (int l = 0; l < 32; ++l) s += buf[lane * 33 + l];
                acc[k >> 5] += s;
            }
            __syncwarp();
        }
    }
};

template <class T>
struct RowLoad {
    const double* row;
    __device__ __forceinline__ T operator()(int k) const { return (T)row[k]; }
};

// a row already converted to FP32 in shared memory (one conversion per coefficient per warp
// instead of one per coefficient per lane)
struct SmemRowF {
    const float* row;
    __device__ __forceinline__ float operator()(int k) const { return row[k]; }
};
// the same as float-float pairs
struct SmemRowFF {
    const ff* row;
    __device__ __forceinline__ ff operator()(int k) const { return row[k]; }
};

// the warp copies an FP64 row into `buf` as FP32
__device__ __forceinline__ void warp_row_to_f32(const double* __restrict__ row, float* buf, int lane) {
    __syncwarp();
    for (int k = lane; k < NC; k += 32) buf[k] = (float)row[k];
    __syncwarp();
}
// ... or an FP32 row
__device__ __forceinline__ void warp_row_f32(const float* __restrict__ row, float* buf, int lane) {
    __syncwarp();
    for (int k = lane; k < NC; k += 32) buf[k] = row[k];
    __syncwarp();
}

// ---- P2M ---------------------------------------------------------------------------------
// rows32: the multipole rows are FP32 (NCP floats per leaf) instead of FP64.  The FP32 kernel
// reads the particles' FP32 leaf-frame records, which hold exactly the values it would compute
// from the FP64 coordinates ((x - c) / h rounded once to FP32), without FP64 arithmetic.
// H: the harmonic basis -- the generated code emits only the (p + 1)^2 free coefficients
// (z exponent <= 1), which are summed and written at their layout positions; the others are
// not computed (the multipole's homogeneous parts are harmonic, Eq. 2, so they are implied).
// f16 (H, FP32 rows): the row's F16 split as well, as tc_split_f16_multi makes it -- the warp
// holds the whole row, so its largest magnitude is one warp reduction away.
template <class T, bool H = false>
__global__ void k_p2m(TreeView tv, double* __restrict__ M, int rows32, F16Rows f16) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw) + threadIdx.y * (32 * 33);
    const int lane = threadIdx.x;
    const int leaf = blockIdx.x * blockDim.y + threadIdx.y;
    if (leaf >= tv.nleaf) return;
    int i0 = tv.leaf_start[leaf], i1 = tv.leaf_start[leaf + 1];
    if (!DAFMM_RANGE(i0, i1, tv.n, kChkLeafRange)) i0 = i1 = 0;
    int a, b, c;
    octmajor_decode(tv.depth, leaf, a, b, c);
    const double cx = tv.x0 + ((double)a + 0.5) * tv.h_leaf;
    const double cy = tv.y0 + ((double)b + 0.5) * tv.h_leaf;
    const double cz = tv.z0 + ((double)c + 0.5) * tv.h_leaf;
    const int r_own = xq_base(i0, leaf) - i0;  // FP32 record of sorted position i: i + r_own
    constexpr int NO = H ? nharm_of(P) : NC;
    constexpr int NJ = (NO + 31) / 32;
    T acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = T(0);
    ChunkSink<T, NJ, NO> sink{sm, lane, acc};
    for (int base = i0; base < i1; base += 32) {
        const int i = base + lane;
        T x = T(0), y = T(0), z = T(0), q = T(0);
        if (i < i1) {
            if constexpr (sizeof(T) == 4) {
                const float4 r = xq_load(tv.xq, i + r_own);
                x = r.x;
                y = r.y;
                z = r.z;
                q = r.w;
            } else {
                x = (T)((tv.x[i] - cx) * tv.inv_h_leaf);
                y = (T)((tv.y[i] - cy) * tv.inv_h_leaf);
                z = (T)((tv.z[i] - cz) * tv.inv_h_leaf);
                q = (T)tv.q[i];
            }
        }
        if constexpr (H) gen::GEN(p2mh)<T>(x, y, z, q, sink);
        else gen::GEN(p2m)<T>(x, y, z, q, sink);
    }
    if (rows32) {
        float* Mf = reinterpret_cast<float*>(M) + (size_t)leaf * NCP;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int k = lane + 32 * j;
            if (k < NO) Mf[H ? harm_full_index(k) : k] = (float)acc[j];
        }
        if constexpr (H && sizeof(T) == 4) {
            if (f16.hi) {
                float mx = 0.f;
#pragma unroll
                for (int j = 0; j < NJ; ++j)
                    if (lane + 32 * j < NO) mx = fmaxf(mx, fabsf((float)acc[j]));
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                int e = 0;
                if (mx > 0.f) frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
                e = e < -120 ? -120 : (e > 120 ? 120 : e);
                const float sc = ldexpf(1.f, -e);
                __half* hi = static_cast<__half*>(f16.hi) + (size_t)leaf * f16.rowlen;
                __half* lo = static_cast<__half*>(f16.lo) + (size_t)leaf * f16.rowlen;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int k = lane + 32 * j;
                    if (k >= f16.rowlen) break;
                    const float f = (k < NO ? (float)acc[j] : 0.f) * sc;
                    const __half h = __float2half_rn(f);
                    hi[k] = h;
                    lo[k] = __float2half_rn(f - __half2float(h));
                }
                if (lane == 0) f16.inv[leaf] = ldexpf(1.f, e);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = lane + 32 * j;
        if (k < NO) M[(size_t)leaf * NCP + (H ? harm_full_index(k) : k)] = (double)acc[j];
    }
}

// ---- M2M / L2L ------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T tab_val(const ShiftTab& t, int e);
template <>
__device__ __forceinline__ double tab_val<double>(const ShiftTab& t, int e) { return t.val[e]; }
template <>
__device__ __forceinline__ float tab_val<float>(const ShiftTab& t, int e) { return t.valf[e]; }

constexpr int SH_ROWS = (NC + 7) / 8;  // output rows per warp (8 warps)

// parents at level lc-1; children at level lc stored octant-major
// Both shifts use the octant structure of Sec. 3.3: the entry (b, a) of the table of child
// octant c is the octant-0 entry times (-1)^popcount(par & c), par = parity pattern of the
// entry.  Summing over the 8 octants first -- the Hadamard transform
//   S_m[a] = sum_c (-1)^popcount(m & c) M_c[a]
// -- turns the 8 signed products per entry into one: parent M[b] = sum_e val_e S_{par_e}[col_e].
// For L2L the transform runs the other way: R_m[b] = sum_{e of parity m} val_e L[col_e], and
// child c receives sum_m (-1)^popcount(m & c) R_m[b].  Table entries are stored per row in
// parity order (tab.rp8).
template <class T>
__device__ __forceinline__ void hadamard8(T (&m)[8]) {
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!(i & h)) {
                const T a = m[i], b = m[i | h];
                m[i] = a + b;
                m[i | h] = a - b;
            }
}

// parents per thread block of the M2M kernels: 8.  The NC output rows of a parent are then
// spread over 32 threads (4 lanes in each of the 8 warps), about NC / 32 rows each; a level of
// 4096 parents spreads over 512 blocks; and the transformed children S[8][8][NCP + 1] (43 KB in
// FP32 at p = 8) leave room for several blocks per SM
template <class T>
constexpr int m2m_parents() {
    return 8;
}
template <class T>
constexpr size_t m2m_smem() {
    return (size_t)8 * m2m_parents<T>() * (NCP + 1) * sizeof(T);
}

// M2M from the children at level lc into the parents at level lc - 1 (uniform tree).  harm:
// harmonic multipoles -- tab is the harmonic M2M table, which reads and writes only the free
// coefficients, so only those are staged and computed.
template <class T>
__global__ void __launch_bounds__(256) k_m2m(ShiftTab tab, int lc, const double* __restrict__ Mc,
                                             double* __restrict__ Mp, int rows32, int harm) {
    constexpr int PP = m2m_parents<T>(), RS = 32 / PP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);  // [8][PP][NCP + 1]
    const int Pc = 1 << (lc - 1);
    const int nparent = Pc * Pc * Pc;
    const int lin0 = blockIdx.x * PP;
    const int NO = harm ? nharm_of(P) : NC;  // coefficients staged and computed per box
    for (int e = threadIdx.x; e < PP * NO; e += 256) {
        const int r = e / NO, j = e - r * NO;
        const int k = harm ? harm_full_index(j) : j;
        const int lin = lin0 + r;
        T m[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const size_t at = (size_t)(c * nparent + lin) * NCP + k;
            m[c] = lin >= nparent ? T(0) : rows32 ? (T)reinterpret_cast<const float*>(Mc)[at] : (T)Mc[at];
        }
        hadamard8(m);
#pragma unroll
        for (int q = 0; q < 8; ++q) S[(q * PP + r) * (NCP + 1) + k] = m[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = lane % PP, sub = lane / PP;
    const int lin = lin0 + r;
    if (lin >= nparent) return;
    const int px = lin % Pc, py = (lin / Pc) % Pc, pz = lin / (Pc * Pc);
    const size_t ob = (size_t)octmajor_index(lc - 1, px, py, pz) * NCP;
    for (int j = w * RS + sub; j < NO; j += 8 * RS) {
        const int b = harm ? harm_full_index(j) : j;
        T acc = T(0);
        for (int e = tab.rowptr[b]; e < tab.rowptr[b + 1]; ++e)
            acc += tab_val<T>(tab, e) * S[(tab.par[e] * PP + r) * (NCP + 1) + tab.col[e]];
        if (rows32) reinterpret_cast<float*>(Mp)[ob + b] = (float)acc;
        else Mp[ob + b] = (double)acc;
    }
}

// the 8 partial sums R_m of row b of the L2L table applied to a local expansion in `src`
template <class T>
__device__ __forceinline__ void l2l_row(const ShiftTab& tab, int b, const T* src, T (&R)[8]) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        T s = T(0);
        for (int e = tab.rp8[8 * b + m]; e < tab.rp8[8 * b + m + 1]; ++e) s += tab_val<T>(tab, e) * src[tab.col[e]];
        R[m] = s;
    }
    hadamard8(R);  // R[c] = what child octant c receives
}

// children at level lc receive L2L of their parent (added to what M2L wrote)
template <class T>
__global__ void __launch_bounds__(256) k_l2l(ShiftTab tab, int lc, const double* __restrict__ Lp,
                                             double* __restrict__ Lc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* src = reinterpret_cast<T*>(smem_raw);  // [32][NCP + 1]
    const int Pc = 1 << (lc - 1);
    const int nparent = Pc * Pc * Pc;
    const int lin0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < 32 * NC; e += 256) {
        const int r = e / NC, k = e - r * NC;
        const int lin = lin0 + r;
        T v = T(0);
        if (lin < nparent) {
            const int px = lin % Pc, py = (lin / Pc) % Pc, pz = lin / (Pc * Pc);
            v = (T)Lp[(size_t)octmajor_index(lc - 1, px, py, pz) * NCP + k];
        }
        src[r * (NCP + 1) + k] = v;
    }
    __syncthreads();
    const int lin = lin0 + lane;
    if (lin >= nparent) return;
    for (int b = w; b < NC; b += 8) {
        T R[8];
        l2l_row(tab, b, src + lane * (NCP + 1), R);
#pragma unroll
        for (int c = 0; c < 8; ++c) Lc[(size_t)(c * nparent + lin) * NCP + b] += (double)R[c];
    }
}

// ---- K generation (Eq. 5 as a matrix per displacement) -------------------------------------
// K^_v[b][a] = coefficient b of sqrt(R) (M2)^a, M2 = (v + u) R, R = 1/|v + u|^2, boxes of width 1.
__device__ void da_mul_block(const MulTab& mt, const double* A, const double* B, double* C) {
    for (int k = threadIdx.x; k < NC; k += blockDim.x) {
        double s = 0.0;
        for (int e = mt.rowptr[k]; e < mt.rowptr[k + 1]; ++e) {
            const ushort2 pr = mt.pairs[e];
            s = fma(A[pr.x], B[pr.y], s);
        }
        C[k] = s;
    }
    __syncthreads();
}

struct SmemStore {
    double* o;
    __device__ __forceinline__ void operator()(int k, double v) const { o[k] = v; }
};

// r0s (optional): block b computes the matrix of the displacement r0s[3 b .. 3 b + 2] (any
// real vector, e.g. along an axis) into slot b of K64, instead of an integer key's
__global__ void __launch_bounds__(256) k_kgen(MulTab mt, double* __restrict__ K64, float* __restrict__ K32,
                                              int key_only, const short* __restrict__ key_list,
                                              const double* __restrict__ r0s) {
    __shared__ double buf[8][NCP];
    const int key = key_only >= 0 ? key_only : (key_list ? key_list[blockIdx.x] : blockIdx.x);
    const int vx = key / 49 - 3, vy = (key / 7) % 7 - 3, vz = key % 7 - 3;
    const int amax = max(abs(vx), max(abs(vy), abs(vz)));
    if (!r0s && amax <= 1) return;  // adjacent boxes never interact through M2L
    double* sR = buf[0];
    double* m2[3] = {buf[1], buf[2], buf[3]};
    double* X = buf[4];
    double* XY = buf[5];
    double* Z0 = buf[6];
    double* Z1 = buf[7];
    const double v[3] = {r0s ? r0s[3 * blockIdx.x] : (double)vx, r0s ? r0s[3 * blockIdx.x + 1] : (double)vy,
                         r0s ? r0s[3 * blockIdx.x + 2] : (double)vz};
    const size_t slot = r0s ? blockIdx.x : (size_t)(key_only >= 0 ? 0 : key);
    const double rho = 1.0 / (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (threadIdx.x == 0) {
        gen::GEN(m2lmap_inv)<double>(v[0], v[1], v[2], rho, SmemStore{X});
        gen::GEN(m2lmap_isq)<double>(v[0], v[1], v[2], rho, SmemStore{sR});
    }
    __syncthreads();
    const double srho = sqrt(rho);
    for (int k = threadIdx.x; k < NC; k += blockDim.x) {
        X[k] *= rho;      // R
        sR[k] *= srho;    // sqrt(R)
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NC; k += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const int km = mt.minus[d * NC + k];
            m2[d][k] = v[d] * X[k] + (km >= 0 ? X[km] : 0.0);
        }
    __syncthreads();
    // monomials (M2)^(a,b,c): X = M2x^a, XY = X M2y^b, Z = XY M2z^c
    for (int k = threadIdx.x; k < NC; k += blockDim.x) X[k] = (k == 0) ? 1.0 : 0.0;
    __syncthreads();
    double* Xn = XY;  // scratch while stepping X
    for (int a = 0; a <= P; ++a) {
        if (a > 0) {
            da_mul_block(mt, X, m2[0], Z0);
            for (int k = threadIdx.x; k < NC; k += blockDim.x) X[k] = Z0[k];
            __syncthreads();
        }
        for (int k = threadIdx.x; k < NC; k += blockDim.x) Xn[k] = X[k];
        __syncthreads();
        for (int b = 0; b <= P - a; ++b) {
            if (b > 0) {
                da_mul_block(mt, Xn, m2[1], Z0);
                for (int k = threadIdx.x; k < NC; k += blockDim.x) Xn[k] = Z0[k];
                __syncthreads();
            }
            double* Zc = Z0;
            double* Zn = Z1;
            for (int k = threadIdx.x; k < NC; k += blockDim.x) Zc[k] = Xn[k];
            __syncthreads();
            for (int c = 0; c <= P - a - b; ++c) {
                if (c > 0) {
                    da_mul_block(mt, Zc, m2[2], Zn);
                    double* t = Zc; Zc = Zn; Zn = t;
                }
                // column alpha = sqrt(R) * Z  -> K[key][beta][alpha]
                const int alpha = da_index(a, b, c);
                double* out = K64 + slot * NC * NCP;
                float* out32 = K32 ? K32 + slot * NC * NCP : nullptr;
                for (int k = threadIdx.x; k < NC; k += blockDim.x) {
                    double s = 0.0;
                    for (int e = mt.rowptr[k]; e < mt.rowptr[k + 1]; ++e) {
                        const ushort2 pr = mt.pairs[e];
                        s = fma(sR[pr.x], Zc[pr.y], s);
                    }
                    out[(size_t)k * NCP + alpha] = s;
                    if (out32) out32[(size_t)k * NCP + alpha] = (float)s;
                }
                __syncthreads();
            }
        }
    }
}

// ---- M2L (SIMT) ----------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ const T* ktab(const double* K64, const float* K32);
template <>
__device__ __forceinline__ const double* ktab<double>(const double* K64, const float*) { return K64; }
template <>
__device__ __forceinline__ const float* ktab<float>(const double*, const float* K32) { return K32; }

// targets: level l, octant blockIdx.y, 32 consecutive parent positions per block
template <class T, class Src>
__global__ void __launch_bounds__(256) k_m2l(const T* __restrict__ K, int l, const Src* __restrict__ M,
                                             double* __restrict__ L, double inv_h) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* src = reinterpret_cast<T*>(smem_raw);  // [32][NCP + 1]
    __shared__ int sidx[32];
    const int Pp = 1 << (l - 1);  // parents per axis
    const int nlin = Pp * Pp * Pp;
    const int oct = blockIdx.y;
    const int lin0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
    const int n_side = 1 << l;
    T acc[SH_ROWS];
#pragma unroll
    for (int j = 0; j < SH_ROWS; ++j) acc[j] = T(0);
    for (int vx = -3 + ox; vx <= 2 + ox; ++vx)
        for (int vy = -3 + oy; vy <= 2 + oy; ++vy)
            for (int vz = -3 + oz; vz <= 2 + oz; ++vz) {
                if (abs(vx) <= 1 && abs(vy) <= 1 && abs(vz) <= 1) continue;
                if (threadIdx.x < 32) {
                    const int lin = lin0 + threadIdx.x;
                    int s = -1;
                    if (lin < nlin) {
                        const int px = lin % Pp, py = (lin / Pp) % Pp, pz = lin / (Pp * Pp);
                        const int tx = 2 * px + ox, ty = 2 * py + oy, tz = 2 * pz + oz;
                        const int sx = tx - vx, sy = ty - vy, sz = tz - vz;
                        if (sx >= 0 && sy >= 0 && sz >= 0 && sx < n_side && sy < n_side && sz < n_side)
                            s = octmajor_index(l, sx, sy, sz);
                    }
                    sidx[threadIdx.x] = s;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < 32 * NC; e += 256) {
                    const int r = e / NC, k = e - r * NC;
                    const int s = sidx[r];
                    src[r * (NCP + 1) + k] = s >= 0 ? (T)M[(size_t)s * NCP + k] : T(0);
                }
                __syncthreads();
                const int key = (vx + 3) * 49 + (vy + 3) * 7 + (vz + 3);
                const T* Kv = K + (size_t)key * NC * NCP;
                const T* srow = src + lane * (NCP + 1);
                const T* kw = Kv + (size_t)w * NCP;  // rows b = w + 8 j
#pragma unroll 1
                for (int a = 0; a < NC; ++a) {
                    const T sv = srow[a];
#pragma unroll
                    for (int j = 0; j < SH_ROWS; ++j)
                        if (w + 8 * j < NC) acc[j] = fma(kw[(size_t)(8 * j) * NCP + a], sv, acc[j]);
                }
                __syncthreads();
            }
    const int lin = lin0 + lane;
    if (lin < nlin) {
        const int t = oct * nlin + lin;
#pragma unroll
        for (int j = 0; j < SH_ROWS; ++j) {
            const int b = w + 8 * j;
            if (b < NC) L[(size_t)t * NCP + b] = (double)acc[j] * inv_h;
        }
    }
}

// ---- M2L by rotation (Sec. 3.4), FP64 -------------------------------------------------------
// K^_v = B_v A_|v| F_v: F_v rotates the source expansion so that v lies on the positive x axis
// (M^(u) = M(Q^T u), Q = Rz(phi) Rx(theta) with theta = atan2(vz, vy), phi = atan2(sqrt(vy^2 +
// vz^2), vx)), A_rho is Eq. 5 along the axis (displacement (rho, 0, 0)), and B_v rotates the
// result back (L(d) = L^(Q d)).  A linear substitution keeps every degree apart; a rotation
// about one axis moves only the other two variables, so it acts on the binary forms of fixed
// exponent of the untouched variable: the form of degree m in (p, q) is multiplied by the
// (m+1) x (m+1) matrix of p -> al p + be q, q -> ga p + de q.  The four substitutions (forward
// about x then z, back about z then x) are tabulated per displacement key; A_rho is sparse:
// column (a, b, c) reaches row (a', b', c') only when b' >= b, c' >= c and both differences are
// even (the axial map depends on y and z through y^2 + z^2 and odd powers of y, z alone).
constexpr int ROT_TSZ = (P + 1) * (P + 2) * (2 * P + 3) / 6;  // sum over m <= P of (m+1)^2

__host__ __device__ constexpr int rot_off(int m) { return m * (m + 1) * (2 * m + 1) / 6; }
// per key: the four substitution matrices (forward x-step, forward z-step, back z-step, back
// x-step), each packed over m = 0..P
__global__ void __launch_bounds__(128) k_rot_tables(double* __restrict__ T) {
    const int key = blockIdx.x;
    const double vx = key / 49 - 3, vy = (key / 7) % 7 - 3, vz = key % 7 - 3;
    const double ryz = sqrt(vy * vy + vz * vz), rho = sqrt(vx * vx + vy * vy + vz * vz);
    const double c1 = ryz > 0.0 ? vy / ryz : 1.0, s1 = ryz > 0.0 ? vz / ryz : 0.0;
    const double c2 = rho > 0.0 ? vx / rho : 1.0, s2 = rho > 0.0 ? ryz / rho : 0.0;
    // (al, be, ga, de) per substitution: old p = al p' + be q', old q = ga p' + de q'
    const double sub[4][4] = {{c1, -s1, s1, c1}, {c2, -s2, s2, c2}, {c2, s2, -s2, c2}, {c1, s1, -s1, c1}};
    for (int e = threadIdx.x; e < 4 * ROT_TSZ; e += blockDim.x) {
        const int w = e / ROT_TSZ, r = e - w * ROT_TSZ;
        int m = 0;
        while (rot_off(m + 1) <= r) ++m;
        const int i = (r - rot_off(m)) / (m + 1), j = (r - rot_off(m)) % (m + 1);
        const double al = sub[w][0], be = sub[w][1], ga = sub[w][2], de = sub[w][3];
        // coefficient of p^(m-i) q^i in (al p + be q)^(m-j) (ga p + de q)^j
        double acc = 0.0;
        for (int k = 0; k <= i; ++k) {  // k from the first factor, i - k from the second
            if (k > m - j || i - k > j) continue;
            double c_a = 1.0, c_b = 1.0;
            for (int t = 0; t < k; ++t) c_a = c_a * (m - j - t) / (t + 1);
            for (int t = 0; t < i - k; ++t) c_b = c_b * (j - t) / (t + 1);
            double pw = c_a * c_b;
            for (int t = 0; t < m - j - k; ++t) pw *= al;
            for (int t = 0; t < k; ++t) pw *= be;
            for (int t = 0; t < j - (i - k); ++t) pw *= ga;
            for (int t = 0; t < i - k; ++t) pw *= de;
            acc += pw;
        }
        T[(size_t)key * 4 * ROT_TSZ + e] = acc;
    }
}

// the axial matrices [nrho][NC][NCP] (dense, from k_kgen) -> their structural non-zeros
__global__ void k_axial_gather(const double* __restrict__ K, const int* __restrict__ rowptr,
                               const unsigned short* __restrict__ col, int nnz, double* __restrict__ val) {
    const int r = blockIdx.x;
    for (int b = threadIdx.x; b < NC; b += blockDim.x)
        for (int e = rowptr[b]; e < rowptr[b + 1]; ++e)
            val[(size_t)r * nnz + e] = K[((size_t)r * NC + b) * NCP + col[e]];
}

// One step of the rotation M2L for the warp: out[k] (=, or += with ACC) sum over the tasks of
// k of tab[offset] * in[index].  Each lane runs its own list of tasks (a precomputed,
// load-balanced share of the step's multiply-adds, whole outputs per lane, padded to a common
// length with tasks that read the zero at in[NC]); task t of lane l is list[32 t + l]:
// x = table offset | last-of-output << 31, y = input index | output index << 16.  Lanes with
// outputs of very different lengths would otherwise run every loop to the longest one, and
// FP64 instructions are this kernel's bound.
// the arithmetic of the rotation M2L: FP64, or float-float (the DAFMM_FF mode)
__device__ __forceinline__ double rot_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff rot_add(ff a, ff b) { return ff_acc(a, b); }
template <class R>
__device__ __forceinline__ R rot_zero() { return R(0.0); }
__device__ __forceinline__ double rot_to_double(double a) { return a; }
__device__ __forceinline__ double rot_to_double(ff a) { return a.to_double(); }

// running sums of a rotation step's output.  FP64: a plain fma chain.  Float-float: a cascaded
// sum (as Ogita, Rump and Oishi's Sum2): each product's high part joins the high sum through
// TwoSum and its rounding error, with the product's low part, joins the low sum; the pair is
// renormalised once per output.  A renormalisation per term (ff_acc) would put about eight
// dependent FP32 operations between consecutive terms of a lane's chain instead of two adds.
struct RotAccD {
    double s = 0.0;
    __device__ __forceinline__ void madd(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
struct RotAccF {
    float hi = 0.f, lo = 0.f;
    // the product enters unnormalised: its rounded high part p through TwoSum, and p's exact
    // rounding error plus the cross terms (a.hi b.lo + a.lo b.hi) into the low sum (13 FP32
    // operations instead of 16 with a renormalised product; the low sum's rounding stays of
    // the order u^2 |a b|)
    __device__ __forceinline__ void madd(ff a, ff b) {
        const float p = mul_rn(a.hi, b.hi);
        const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, mul_rn(a.lo, b.hi));
        const ff t = two_sum(hi, p);
        hi = t.hi;
        lo += t.lo + e;
    }
    __device__ __forceinline__ ff get() const { return fast_two_sum(hi, lo); }
};
template <class R>
struct RotAcc;
template <>
struct RotAcc<double> {
    using type = RotAccD;
};
template <>
struct RotAcc<ff> {
    using type = RotAccF;
};

template <bool ACC, class R>
__device__ __forceinline__ void rot_step(const uint2* __restrict__ list, int len, const R* __restrict__ tab,
                                         const R* in, R* out, int lane) {
    typename RotAcc<R>::type s;
#pragma unroll 4
    for (int t = 0; t < len; ++t) {
        const uint2 w = list[32 * t + lane];
        if (DAFMM_IN(w.y & 0xffffu, NC + 1, kChkRotTask)) s.madd(tab[w.x & 0x7fffffffu], in[w.y & 0xffffu]);
        if (w.x >> 31) {
            const int k = (int)(w.y >> 16);
            if (DAFMM_IN(k, NC, kChkRotTask)) {
                if (ACC) out[k] = rot_add(out[k], s.get());
                else out[k] = s.get();
            }
            s = typename RotAcc<R>::type();
        }
    }
}

// task lists of the rotation M2L: x-step (substitution about x), z-step, axial matrix
struct RotLists {
    const uint2* x;
    const uint2* z;
    const uint2* a;
    int lx, lz, la;
};

// the harmonic form of the rotation (harmonic task lists): the steps that restore a vector's
// coefficients of z exponent >= 2 from its free ones by Laplace's equation (step s sets
// V[i] = w1 V[i1] + w2 V[i2]; those of z exponent c at [cst[c], cst[c + 1]))
struct RotHarm {
    const int4* step;
    const double2* w;
    int cst[kMaxOrder + 3];
};

__device__ __forceinline__ double rot_axpby(double w1, double a, double w2, double b) { return fma(w1, a, w2 * b); }
__device__ __forceinline__ ff rot_axpby(double w1, ff a, double w2, ff b) {
    return ff_add(ff_mul(ff(w1), a), ff_mul(ff(w2), b));
}

// the warp restores V's coefficients of z exponent >= 2, level by level
template <class R>
__device__ __forceinline__ void rot_expand(R* V, const RotHarm& hm, int lane) {
#pragma unroll 1
    for (int c = 2; c <= P; ++c) {
        for (int s = hm.cst[c] + lane; s < hm.cst[c + 1]; s += 32) {
            const int4 st = hm.step[s];
            const double2 w = hm.w[s];
            V[st.x] = rot_axpby(w.x, V[st.y], w.y, V[st.z]);
        }
        __syncwarp();
    }
}

// a source row into the work vector: FP64 rows, or (float-float) the rows' FP32 high and low
// parts, split once per evaluation
__device__ __forceinline__ void rot_load(double* X, const double* M, const float*, const float*, size_t row, int lane) {
    for (int k = lane; k < NC; k += 32) X[k] = M[row + k];
}
__device__ __forceinline__ void rot_load(ff* X, const double*, const float* Mh, const float* Ml, size_t row, int lane) {
    for (int k = lane; k < NC; k += 32) X[k] = ff(Mh[row + k], Ml[row + k]);
}

// one well-separated pair for the warp: S += B_v A_|v| F_v Ms (T: the key's four substitution
// tables, av: the axial matrix of its length; X, Y: work vectors with X[NC] = Y[NC] = 0; the
// source row at `row` of M, or of Mh / Ml in float-float)
// HARM: harmonic task lists (free outputs only), the vector restored before the last x-step
template <class R, bool HARM>
__device__ __forceinline__ void rot_pair(const R* __restrict__ T, const R* __restrict__ av, const RotLists& rl,
                                         const double* __restrict__ M, const float* __restrict__ Mh,
                                         const float* __restrict__ Ml, size_t row, R* X, R* Y, R* S, int lane,
                                         const RotHarm& hm) {
    __syncwarp();
    rot_load(X, M, Mh, Ml, row, lane);
    __syncwarp();
    rot_step<false>(rl.x, rl.lx, T, X, Y, lane);  // forward, about x
    __syncwarp();
    rot_step<false>(rl.z, rl.lz, T + ROT_TSZ, Y, X, lane);  // forward, about z
    __syncwarp();
    rot_step<false>(rl.a, rl.la, av, X, Y, lane);  // Eq. 5 on the axis
    __syncwarp();
    rot_step<false>(rl.z, rl.lz, T + 2 * ROT_TSZ, Y, X, lane);  // back, about z
    __syncwarp();
    if constexpr (HARM) rot_expand<R>(X, hm, lane);  // the x-step reads every z exponent
    rot_step<true>(rl.x, rl.lx, T + 3 * ROT_TSZ, X, S, lane);  // back, about x, into the sums
}

// the per-warp work vectors of k_m2l_rot
template <class R>
struct RotBuf {
    R v[3][NCP + 1];
};

// R = double: FP64.  R = ff: float-float, the source rows from their FP32 split parts.  The work
// vectors are in shared memory; the task lists (the same for every pair) are read through the
// L1 cache (copies of them in shared memory cost the float-float kernel a quarter of its
// resident warps and gained nothing: measured 73.7 -> 75.5 ms at level 5, N = 1e6, p = 8).
template <class R, bool HARM>
__global__ void __launch_bounds__(256, 2) k_m2l_rot(const R* __restrict__ Ttab, const int* __restrict__ krho,
                                                    RotLists rl, const R* __restrict__ aval, int annz, int l,
                                                    const double* __restrict__ M, const float* __restrict__ Mh,
                                                    const float* __restrict__ Ml, double* __restrict__ L,
                                                    double inv_h, const __grid_constant__ RotHarm hm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ RotBuf<R> bufs[8];
    const int Pp = 1 << (l - 1), P3 = Pp * Pp * Pp, n_side = 1 << l;
    const int t = blockIdx.x * 8 + w;  // target box, octant-major
    if (t >= 8 * P3) return;
    const int oct = t / P3, lin = t - oct * P3;
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
    const int tx = 2 * (lin % Pp) + ox, ty = 2 * ((lin / Pp) % Pp) + oy, tz = 2 * (lin / (Pp * Pp)) + oz;
    R* X = bufs[w].v[0];
    R* Y = bufs[w].v[1];
    R* S = bufs[w].v[2];
    for (int k = lane; k <= NCP; k += 32) {
        X[k] = rot_zero<R>();  // X[NC], Y[NC]: the zero that padding tasks read
        Y[k] = rot_zero<R>();
        S[k] = rot_zero<R>();
    }
    for (int vx = -3 + ox; vx <= 2 + ox; ++vx)
        for (int vy = -3 + oy; vy <= 2 + oy; ++vy)
            for (int vz = -3 + oz; vz <= 2 + oz; ++vz) {
                if (abs(vx) <= 1 && abs(vy) <= 1 && abs(vz) <= 1) continue;
                const int sx = tx - vx, sy = ty - vy, sz = tz - vz;
                if (sx < 0 || sy < 0 || sz < 0 || sx >= n_side || sy >= n_side || sz >= n_side) continue;
                const int key = (vx + 3) * 49 + (vy + 3) * 7 + (vz + 3);
                rot_pair<R, HARM>(Ttab + (size_t)key * 4 * ROT_TSZ, aval + (size_t)krho[key] * annz, rl, M, Mh, Ml,
                                  (size_t)octmajor_index(l, sx, sy, sz) * NCP, X, Y, S, lane, hm);
            }
    __syncwarp();
    if constexpr (HARM) rot_expand<R>(S, hm, lane);  // the sums' coefficients of z exponent >= 2
    for (int k = lane; k < NC; k += 32) L[(size_t)t * NCP + k] = rot_to_double(S[k]) * inv_h;
}

// the float-float split of FP64 rows (n values): hi = fl32(v), lo = fl32(v - hi)
__global__ void k_split_ff(const double* __restrict__ a, float* __restrict__ hi, float* __restrict__ lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const ff v(a[i]);
        hi[i] = v.hi;
        lo[i] = v.lo;
    }
}

// the same for the targets tg[g0 .. g1) of one (level, octant) group of an adaptive tree (V-list
// sources through the parent's colleagues, as in k_m2l_a); one warp per target
template <bool HARM>
__global__ void __launch_bounds__(256, 2) k_m2l_rot_a(const double* __restrict__ Ttab, const int* __restrict__ krho,
                                                      RotLists rl, const double* __restrict__ aval, int annz,
                                                      AdaptiveView av, const int* __restrict__ tg,
                                                      const int* __restrict__ grp_ptr, int grp0,
                                                      const double* __restrict__ M, double* __restrict__ L,
                                                      const __grid_constant__ RotHarm hm) {
    __shared__ double sbuf[8][3][NCP + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int oct = blockIdx.y;
    const int g0 = grp_ptr[grp0 + oct], g1 = grp_ptr[grp0 + oct + 1];
    const int ti = g0 + blockIdx.x * 8 + w;
    if (ti >= g1 || !DAFMM_RANGE(g0, g1, av.nbox, kChkListPtr)) return;
    if (!DAFMM_IN(tg[ti], av.nbox, kChkBoxIndex) || !DAFMM_IN(av.parent[tg[ti]], av.nbox, kChkBoxIndex)) return;
    const int t = tg[ti], P = av.parent[t];
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
    double* X = sbuf[w][0];
    double* Y = sbuf[w][1];
    double* S = sbuf[w][2];
    for (int k = lane; k <= NCP; k += 32) {
        X[k] = 0.0;
        Y[k] = 0.0;
        S[k] = 0.0;
    }
    for (int vx = -3 + ox; vx <= 2 + ox; ++vx)
        for (int vy = -3 + oy; vy <= 2 + oy; ++vy)
            for (int vz = -3 + oz; vz <= 2 + oz; ++vz) {
                if (abs(vx) <= 1 && abs(vy) <= 1 && abs(vz) <= 1) continue;
                const int dx = ox - vx, dy = oy - vy, dz = oz - vz;  // = 2a + sc
                const int scx = dx & 1, scy = dy & 1, scz = dz & 1;
                const int ax = (dx - scx) >> 1, ay = (dy - scy) >> 1, az = (dz - scz) >> 1;
                const int Q = av.colleague[27 * P + (ax + 1) * 9 + (ay + 1) * 3 + (az + 1)];
                if (Q < 0 || !DAFMM_IN(Q, av.nbox, kChkBoxIndex)) continue;
                const int sb = av.child[8 * Q + (scx | (scy << 1) | (scz << 2))];
                if (sb < 0 || !DAFMM_IN(sb, av.nbox, kChkBoxIndex)) continue;
                const int key = (vx + 3) * 49 + (vy + 3) * 7 + (vz + 3);
                rot_pair<double, HARM>(Ttab + (size_t)key * 4 * ROT_TSZ, aval + (size_t)krho[key] * annz, rl, M,
                                       nullptr, nullptr, (size_t)sb * NCP, X, Y, S, lane, hm);
            }
    __syncwarp();
    if constexpr (HARM) rot_expand<double>(S, hm, lane);  // the sums' coefficients of z exponent >= 2
    const double inv_h = 1.0 / av.geom[t].w;  // the target box's width (each tree has its own)
    for (int k = lane; k < NC; k += 32) L[(size_t)t * NCP + k] = S[k] * inv_h;
}

// float-float copies of the rotation tables and axial values (n doubles each)
__global__ void k_to_ff(const double* __restrict__ a, ff* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = ff(a[i]);
}

// ---- leaves: P2P over the 27 neighbours + L2P --------------------------------------------------
// 1/sqrt(x) of the PTX instruction rsqrt.approx.ftz.f32 (relative error about 2^-23, the
// size of an FP32 rounding, so no Newton step is needed)
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// the same, and 0 for x below the smallest normal float, which covers coincident points
// (r = 0 contributes nothing, as everywhere else)
__device__ __forceinline__ float rsqrt_or_zero(float x) {
    const float y = rsqrt_approx(x);
    return x >= 1.17549435e-38f ? y : 0.f;
}

// Shared-memory source list of the near field, in the target leaf's frame: pair p of the list
// (records 2p and 2p + 1) occupies four float4s from buf[4p]:
//   (X, X', Y, Y')  (Z, Z', Q, Q')      offsets and charges rounded to FP32
//   (x, x', y, y')  (z, z', q, q')      their FP32 remainders
__device__ __forceinline__ void list_store(float4* buf, int j, float X, float Y, float Z, float Q, float xl,
                                           float yl, float zl, float ql) {
    float* f = reinterpret_cast<float*>(buf) + 16 * (j >> 1) + (j & 1);
    f[0] = X;
    f[2] = Y;
    f[4] = Z;
    f[6] = Q;
    f[8] = xl;
    f[10] = yl;
    f[12] = zl;
    f[14] = ql;
}
// a record that adds exactly nothing (q = 0, far from every target: finite 1/r, no guard needed)
__device__ __forceinline__ void list_store_null(float4* buf, int j) {
    list_store(buf, j, 4096.f, 4096.f, 4096.f, 0.f, 0.f, 0.f, 0.f, 0.f);
}

// (H, L) = hi + lo shifted by d with the rounding of hi + d moved into L (Fast2Sum: exact when
// |d| >= |hi| or d = 0, which holds for the integer leaf offsets d in {-1, 0, 1} of a uniform
// tree and |hi| <= 1/2)
__device__ __forceinline__ void shift_exact(float hi, float lo, float d, float& H, float& L) {
    H = hi + d;
    L = lo + (hi - (H - d));
}
// (H, L) = (hi + lo) * r + (oh + ol) for a power of two r, with the rounding of hi * r + oh
// moved into L (TwoSum: exact for any ordering of the two terms)
__device__ __forceinline__ void scale_shift_exact(float hi, float lo, float r, float oh, float ol, float& H,
                                                  float& L) {
    const float a = hi * r;  // exact
    H = a + oh;
    const float bb = H - a;
    const float err = (a - (H - bb)) + (oh - bb);
    L = fmaf(lo, r, err + ol);
}

// pairs of the list per close-pair vote (the unguarded passes)
#ifndef DAFMM_P2P_GROUP
#define DAFMM_P2P_GROUP 2
#endif

// a pair closer than this (in leaf widths of the target's leaf) takes the remainders of its
// offsets into its difference: beyond it, T - S alone is within a few FP32 roundings of the
// difference's own size (the remainders are below 2^-23 leaf widths)
constexpr float kCloseR2 = 0.01f;

// list pairs [p0, p1) acting on the target t = T + tl (T: rounded offsets, tl: remainders,
// in the list's frame), both halves of every step in one packed FP32x2 instruction: per half
//   e = T - S  (+ (tl - sl) when |e| < 0.1),  r2 = fma(ex, ex, fma(ey, ey, ez ez)),
//   qr = q / r,  qr3 = qr / r^2,
// and the halves accumulate separately in P (potential) and X, Y, Z (field without its sign
// convention).  e carries the difference of the two particles to a few FP32 roundings of
// itself however close they are: pairs closer than 0.1 leaf widths -- rare, so the remainders
// are loaded and added only in an iteration where a lane of the warp has one -- take the
// remainders.  GUARD (the target's own leaf, which holds the target and any coincident
// particles) always takes them and gives r = 0 no contribution; without it r2 starts from the
// smallest normal float, so distinct particles -- which never coincide across leaves --
// always give a finite 1/r.
// one pair of the list: its difference e (T - S, plus the remainders for the target's own
// leaf) and r^2
template <bool GUARD>
__device__ __forceinline__ void p2p_diff(const float4* __restrict__ buf, int p, float2 tx, float2 ty, float2 tz,
                                         float2 lx, float2 ly, float2 lz, float2& ex, float2& ey, float2& ez,
                                         float2& r2, float2& q) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float4 A = buf[4 * p], B = buf[4 * p + 1];
    ex = __ffma2_rn(make_float2(A.x, A.y), m1, tx);
    ey = __ffma2_rn(make_float2(A.z, A.w), m1, ty);
    ez = __ffma2_rn(make_float2(B.x, B.y), m1, tz);
    q = make_float2(B.z, B.w);
    if (GUARD) {
        const float4 C = buf[4 * p + 2], D = buf[4 * p + 3];
        ex = __fadd2_rn(ex, __ffma2_rn(make_float2(C.x, C.y), m1, lx));
        ey = __fadd2_rn(ey, __ffma2_rn(make_float2(C.z, C.w), m1, ly));
        ez = __fadd2_rn(ez, __ffma2_rn(make_float2(D.x, D.y), m1, lz));
        r2 = __fmul2_rn(ez, ez);
    } else {
        r2 = __ffma2_rn(ez, ez, make_float2(1.17549435e-38f, 1.17549435e-38f));
    }
    r2 = __ffma2_rn(ey, ey, r2);
    r2 = __ffma2_rn(ex, ex, r2);
}

// a pair closer than 0.1 leaf widths takes the remainders into its difference (halves whose
// r^2 is below kCloseR2; the others keep T - S)
__device__ __forceinline__ void p2p_close(const float4* __restrict__ buf, int p, float2 lx, float2 ly, float2 lz,
                                          float2& ex, float2& ey, float2& ez, float2& r2) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const bool cx = r2.x < kCloseR2, cy = r2.y < kCloseR2;
    const float4 C = buf[4 * p + 2], D = buf[4 * p + 3];
    const float2 fx = __fadd2_rn(ex, __ffma2_rn(make_float2(C.x, C.y), m1, lx));
    const float2 fy = __fadd2_rn(ey, __ffma2_rn(make_float2(C.z, C.w), m1, ly));
    const float2 fz = __fadd2_rn(ez, __ffma2_rn(make_float2(D.x, D.y), m1, lz));
    if (cx) {
        ex.x = fx.x;
        ey.x = fy.x;
        ez.x = fz.x;
    }
    if (cy) {
        ex.y = fx.y;
        ey.y = fy.y;
        ez.y = fz.y;
    }
    r2 = __ffma2_rn(ez, ez, make_float2(1.17549435e-38f, 1.17549435e-38f));
    r2 = __ffma2_rn(ey, ey, r2);
    r2 = __ffma2_rn(ex, ex, r2);
}

// the pair's terms into the sums
template <bool GUARD>
__device__ __forceinline__ void p2p_acc(float2 ex, float2 ey, float2 ez, float2 r2, float2 q, float2& P, float2& X,
                                        float2& Y, float2& Z) {
    const float2 ir = GUARD ? make_float2(rsqrt_or_zero(r2.x), rsqrt_or_zero(r2.y))
                            : make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    const float2 qr = __fmul2_rn(q, ir);
    const float2 qr3 = __fmul2_rn(qr, __fmul2_rn(ir, ir));
    P = __fadd2_rn(P, qr);
    X = __ffma2_rn(qr3, ex, X);
    Y = __ffma2_rn(qr3, ey, Y);
    Z = __ffma2_rn(qr3, ez, Z);
}

// list pairs [p0, p1) acting on the target t = T + tl (T: rounded offsets, tl: remainders,
// in the list's frame), both halves of every step in one packed FP32x2 instruction: per half
//   e = T - S  (+ (tl - sl) when |e| < 0.1),  r2 = fma(ex, ex, fma(ey, ey, ez ez)),
//   qr = q / r,  qr3 = qr / r^2,
// and the halves accumulate separately in P (potential) and X, Y, Z (field without its sign
// convention).  e carries the difference of the two particles to a few FP32 roundings of
// itself however close they are: pairs closer than 0.1 leaf widths -- rare -- take the
// remainders, loaded and added only for a group of four pairs in which a lane of the warp has
// one (one vote per group keeps the group's arithmetic in one stretch of code).  GUARD
// (the target's own leaf, which holds the target and any coincident particles) always takes
// them and gives r = 0 no contribution; without it r2 starts from the smallest normal float,
// so distinct particles -- which never coincide across leaves -- always give a finite 1/r.
template <bool GUARD>
__device__ __forceinline__ void p2p_pairs(const float4* __restrict__ buf, int p0, int p1, float2 tx, float2 ty,
                                          float2 tz, float2 lx, float2 ly, float2 lz, float2& P, float2& X,
                                          float2& Y, float2& Z) {
    int p = p0;
    if (!GUARD) {
        constexpr int G = DAFMM_P2P_GROUP;
        for (; p + G <= p1; p += G) {
            float2 ex[G], ey[G], ez[G], r2[G], q[G];
            float rmin = 3.0e38f;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                p2p_diff<false>(buf, p + k, tx, ty, tz, lx, ly, lz, ex[k], ey[k], ez[k], r2[k], q[k]);
                rmin = fminf(rmin, fminf(r2[k].x, r2[k].y));
            }
            if (__any_sync(__activemask(), rmin < kCloseR2)) {
#pragma unroll
                for (int k = 0; k < G; ++k) p2p_close(buf, p + k, lx, ly, lz, ex[k], ey[k], ez[k], r2[k]);
            }
#pragma unroll
            for (int k = 0; k < G; ++k) p2p_acc<false>(ex[k], ey[k], ez[k], r2[k], q[k], P, X, Y, Z);
        }
    }
#pragma unroll 4
    for (; p < p1; ++p) {
        float2 ex, ey, ez, r2, q;
        p2p_diff<GUARD>(buf, p, tx, ty, tz, lx, ly, lz, ex, ey, ez, r2, q);
        if (!GUARD && __any_sync(__activemask(), r2.x < kCloseR2 || r2.y < kCloseR2))
            p2p_close(buf, p, lx, ly, lz, ex, ey, ez, r2);
        p2p_acc<GUARD>(ex, ey, ez, r2, q, P, X, Y, Z);
    }
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

// compensated (hi, lo) sums of the near field: FP32 partial sums over at most 128 sources are
// folded into them, so that long neighbour lists keep FP32-level error
struct CompSums {
    float ph = 0.f, pl = 0.f, xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f, zh = 0.f, zl = 0.f;
};


// ---- float-float near field (the DAFMM_FF mode) ----
// a cascaded float-float sum (as Ogita, Rump and Oishi's Sum2): the high parts through TwoSum,
// their rounding errors and the low parts into the low sum; renormalised once, by get()
struct FFCasc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(ff v) {
        const ff t = two_sum(hi, v.hi);
        hi = t.hi;
        lo += t.lo + v.lo;
    }
    __device__ __forceinline__ ff get() const { return fast_two_sum(hi, lo); }
};
struct FFSums {
    FFCasc p, x, y, z;
};

// the difference (T + tl) - (S + sl) in float-float: TwoSum of the rounded parts (exact), the
// remainders' difference (below 2^-23 leaf widths, one FP32 rounding) added, renormalised
__device__ __forceinline__ ff ff_diff(float T, float tl, float S, float sl) {
    const ff d = two_sum(T, -S);
    return two_sum(d.hi, d.lo + (tl - sl));
}

// list records [2 pa, 2 pe) acting on the target t = T + tl, every step in float-float (about
// 48 bits): e as above, r^2 = e.e, 1/r by the Newton-refined float-float 1/sqrt, q (rounded
// charge plus its remainder) / r and q / r^3 into float-float sums.  The records below 2 pown
// are the target's own leaf: a pair at r = 0 (the target itself, coincident particles) adds
// nothing; elsewhere r^2 is kept at least the smallest normal float.
__device__ __forceinline__ void p2p_segment_ff(const float4* __restrict__ buf, int pa, int pe, int pown, float tx,
                                               float ty, float tz, float tlx, float tly, float tlz, FFSums& acc) {
#pragma unroll 1
    for (int p = pa; p < pe; ++p) {
        const float4 A = buf[4 * p], B = buf[4 * p + 1], C = buf[4 * p + 2], D = buf[4 * p + 3];
        const bool own = p < pown;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const ff ex = ff_diff(tx, tlx, h ? A.y : A.x, h ? C.y : C.x);
            const ff ey = ff_diff(ty, tly, h ? A.w : A.z, h ? C.w : C.z);
            const ff ez = ff_diff(tz, tlz, h ? B.y : B.x, h ? D.y : D.x);
            ff r2 = ff_acc(ff_acc(ff_mul(ex, ex), ff_mul(ey, ey)), ff_mul(ez, ez));
            if (own && r2.hi == 0.f) continue;
            r2.hi = fmaxf(r2.hi, 1.17549435e-38f);
            const ff ir = ff_rsqrt(r2);
            const ff qr = ff_mul(ff(h ? B.w : B.z, h ? D.w : D.z), ir);
            const ff qr3 = ff_mul(qr, ff_mul(ir, ir));
            acc.p.add(qr);
            acc.x.add(ff_mul(qr3, ex));
            acc.y.add(ff_mul(qr3, ey));
            acc.z.add(ff_mul(qr3, ez));
        }
    }
}

__device__ __forceinline__ ff ff_shfl_down(ff v, int d) {
    return ff(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}

// records per shared-memory segment of the neighbour list (per warp; 32 bytes each)
#ifndef DAFMM_LEAF_SEG
#define DAFMM_LEAF_SEG 128
#endif
constexpr int kLeafSeg = DAFMM_LEAF_SEG;
// blocks per SM the uniform FP32 leaf kernel is compiled for (its register budget)
#ifndef DAFMM_LEAF_MINB
#define DAFMM_LEAF_MINB 8
#endif

// list pairs (two sources each) per FP32 partial sum of the near field: 64 pairs, 128 sources
// (64 in each packed half) -- one fold per list segment of kLeafSeg = 128 records
constexpr int kFoldPairs = 64;

// the pairwise sums of one segment of the list: pairs [pa, pe) for this lane's target, those
// below pown from the target's own leaf (guarded), FP32 partial sums over at most kFoldPairs
// pairs folded into the compensated sums
__device__ __forceinline__ void p2p_segment(const float4* __restrict__ buf, int pa, int pe, int pown, float2 tx,
                                            float2 ty, float2 tz, float2 lx, float2 ly, float2 lz, CompSums& cs) {
    for (int pb = pa; pb < pe; pb += kFoldPairs) {
        const int pc = min(pe, pb + kFoldPairs);
        const int pm = max(pb, min(pc, pown));
        float2 P = make_float2(0.f, 0.f), X = P, Y = P, Z = P;
        if (pb < pm) p2p_pairs<true>(buf, pb, pm, tx, ty, tz, lx, ly, lz, P, X, Y, Z);
        if (pm < pc) p2p_pairs<false>(buf, pm, pc, tx, ty, tz, lx, ly, lz, P, X, Y, Z);
        two_sum_add(cs.ph, cs.pl, P.x + P.y);
        two_sum_add(cs.xh, cs.xl, X.x + X.y);
        two_sum_add(cs.yh, cs.yl, Y.x + Y.y);
        two_sum_add(cs.zh, cs.zl, Z.x + Z.y);
    }
}

// the upper half-warp's sums join the lower one's (passes whose sources were split between
// the half-warps)
__device__ __forceinline__ void join_halves(CompSums& cs) {
    float v[8] = {cs.ph, cs.pl, cs.xh, cs.xl, cs.yh, cs.yl, cs.zh, cs.zl};
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __shfl_down_sync(0xffffffffu, v[j], 16);
    two_sum_add(cs.ph, cs.pl, v[0]);
    cs.pl += v[1];
    two_sum_add(cs.xh, cs.xl, v[2]);
    cs.xl += v[3];
    two_sum_add(cs.yh, cs.yl, v[4]);
    cs.yl += v[5];
    two_sum_add(cs.zh, cs.zl, v[6]);
    cs.zl += v[7];
}

// the neighbour slot (0..26, slot 13 = the leaf itself) held by lane k of the list: the leaf
// itself first, so that its records -- the only ones that can coincide with a target -- form
// the guarded head of the list
__device__ __forceinline__ int own_first_slot(int k) { return k == 0 ? 13 : (k <= 13 ? k - 1 : k); }

template <class T>
__global__ void __launch_bounds__(128, std::is_same<T, float>::value ? DAFMM_LEAF_MINB : (std::is_same<T, ff>::value ? 4 : 8))
k_leaf(TreeView tv, const double* __restrict__ Lleaf,
                                              double* __restrict__ phi, double* __restrict__ field) {
    const int lane = threadIdx.x;
    const int leaf = blockIdx.x * blockDim.y + threadIdx.y;
    if (leaf >= tv.nleaf) return;
    int i0 = tv.leaf_start[leaf], i1 = tv.leaf_start[leaf + 1];
    if (!DAFMM_RANGE(i0, i1, tv.n, kChkLeafRange)) i0 = i1 = 0;
    int a, b, c;
    octmajor_decode(tv.depth, leaf, a, b, c);
    const int nside = 1 << tv.depth;
    const double cx = tv.x0 + ((double)a + 0.5) * tv.h_leaf;
    const double cy = tv.y0 + ((double)b + 0.5) * tv.h_leaf;
    const double cz = tv.z0 + ((double)c + 0.5) * tv.h_leaf;
    const double* Lrow = Lleaf ? Lleaf + (size_t)leaf * NCP : nullptr;
    __shared__ float s_lrow[4][NCP];  // per warp: the leaf's local expansion in FP32
    __shared__ ff s_lrow_ff[std::is_same<T, ff>::value ? 4 : 1][std::is_same<T, ff>::value ? NCP : 1];
    if constexpr (std::is_same<T, ff>::value) {  // ... or in float-float
        if (Lrow) {
            __syncwarp();
            for (int k = lane; k < NC; k += 32) s_lrow_ff[threadIdx.y][k] = ff(Lrow[k]);
            __syncwarp();
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (Lrow) {
            if (tv.locals_f32) {  // the row is FP32 already (NCP floats per leaf)
                const float* Lf = reinterpret_cast<const float*>(Lleaf) + (size_t)leaf * NCP;
                __syncwarp();
                for (int k = lane; k < NC; k += 32) s_lrow[threadIdx.y][k] = Lf[k];
                __syncwarp();
            } else {
                warp_row_to_f32(Lrow, s_lrow[threadIdx.y], lane);
            }
        }
    }
    // FP32: the 27 neighbour leaves' particle ranges, one per lane (empty outside the domain),
    // and the first FP32 record of each, laid end to end as one list: the leaf's own records
    // first (lane 0), completed to an even count by a null record; lane k's neighbour starts
    // at nb_off (exclusive scan of the counts over the lanes), nb_tot records in all, the
    // first own_pairs pairs the leaf's own
    int nb_n = 0, nb_r0 = 0, nb_off = 0, nb_tot = 0, n_own = 0, own_pad = 0, own_pairs = 0;
    if constexpr (!std::is_same<T, double>::value) {
        int nb_s0 = 0, nb_s1 = 0;
        if (lane < 27) {
            const int slot = own_first_slot(lane);
            const int dx = slot % 3 - 1, dy = (slot / 3) % 3 - 1, dz = slot / 9 - 1;
            const int na = a + dx, nb = b + dy, nc2 = c + dz;
            if (na >= 0 && nb >= 0 && nc2 >= 0 && na < nside && nb < nside && nc2 < nside) {
                const int nl = octmajor_index(tv.depth, na, nb, nc2);
                nb_s0 = tv.leaf_start[nl];
                nb_s1 = tv.leaf_start[nl + 1];
                if (!DAFMM_RANGE(nb_s0, nb_s1, tv.n, kChkLeafRange)) nb_s0 = nb_s1 = 0;
                nb_r0 = xq_base(nb_s0, nl);
            }
        }
        nb_n = nb_s1 - nb_s0;
        nb_off = nb_n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, nb_off, d);
            if (lane >= d) nb_off += v;
        }
        n_own = __shfl_sync(0xffffffffu, nb_n, 0);
        own_pad = n_own & 1;
        nb_tot = __shfl_sync(0xffffffffu, nb_off, 31) + own_pad;
        nb_off -= nb_n;
        if (lane > 0) nb_off += own_pad;
        own_pairs = (n_own + 1) >> 1;
    }
    const int r_own = xq_base(i0, leaf) - i0;  // record of sorted position t: t + r_own
    for (int base = i0; base < i1; base += 32) {
        // FP32: a pass of at most 16 targets splits the sources between the two half-warps,
        // lane l and lane l + 16 taking the same target
        const int m = min(32, i1 - base);
        const bool split = !std::is_same<T, double>::value && m <= 16;
        const int tl = split ? (lane & 15) : lane;
        const int t = base + tl;
        const bool valid = tl < m && (!split || lane < 16);  // the lanes that write
        const int tt = tl < m ? t : i0;
        double fphi = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;  // near field, physical units
        if constexpr (std::is_same<T, double>::value) {
            const double xt = tv.x[tt], yt = tv.y[tt], zt = tv.z[tt];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int na = a + dx, nb = b + dy, nc2 = c + dz;
                        if (na < 0 || nb < 0 || nc2 < 0 || na >= nside || nb >= nside || nc2 >= nside) continue;
                        const int nl = octmajor_index(tv.depth, na, nb, nc2);
                        int s0 = tv.leaf_start[nl], s1 = tv.leaf_start[nl + 1];
                        if (!DAFMM_RANGE(s0, s1, tv.n, kChkLeafRange)) s0 = s1 = 0;
                        for (int s = s0; s < s1; ++s) {
                            const double ex = xt - tv.x[s], ey = yt - tv.y[s], ez = zt - tv.z[s];
                            const double r2 = ex * ex + ey * ey + ez * ez;
                            if (r2 > 0.0) {
                                const double ir = rsqrt(r2);
                                const double qr = tv.q[s] * ir;
                                const double qr3 = qr * ir * ir;
                                fphi += qr;
                                fx += qr3 * ex; fy += qr3 * ey; fz += qr3 * ez;
                            }
                        }
                    }
        } else {
            const float4* xl = tv.xq + xq_records(tv.n, tv.nleaf);  // the remainder records
            const float4 pt = xq_load(tv.xq, tt + r_own), pl = xq_load(xl, tt + r_own);
            CompSums cs;
            FFSums fs;
            // The neighbours' records are copied into one shared-memory list, shifted into this
            // leaf's frame (source + neighbour offset, in leaf widths, exactly: the rounding of
            // the shift joins the remainder), in segments of up to kLeafSeg records; the pairwise
            // sum then runs over the whole list.  A pass of at most 16 targets gives each
            // half-warp half of the pairs.
            __shared__ __align__(16) float4 s_list[4][2 * kLeafSeg];
            float4* buf = s_list[threadIdx.y];
            const int g = split ? lane >> 4 : 0;
            const float2 tx2 = make_float2(pt.x, pt.x), ty2 = make_float2(pt.y, pt.y),
                         tz2 = make_float2(pt.z, pt.z);
            const float2 lx2 = make_float2(pl.x, pl.x), ly2 = make_float2(pl.y, pl.y),
                         lz2 = make_float2(pl.z, pl.z);
            for (int seg0 = 0; seg0 < nb_tot; seg0 += kLeafSeg) {
                const int segn = min(kLeafSeg, nb_tot - seg0), seg1 = seg0 + segn;
                __syncwarp();  // the previous segment is no longer read
                // the neighbours whose records fall into this segment
                unsigned ov = __ballot_sync(0xffffffffu, lane < 27 && nb_n > 0 && nb_off < seg1 && nb_off + nb_n > seg0);
                while (ov) {
                    const int k = __ffs(ov) - 1;
                    ov &= ov - 1;
                    const int o = __shfl_sync(0xffffffffu, nb_off, k), n = __shfl_sync(0xffffffffu, nb_n, k);
                    const int r0 = __shfl_sync(0xffffffffu, nb_r0, k);
                    const int slot = own_first_slot(k);
                    const int lo = max(o, seg0), hi = min(o + n, seg1);
                    const float dx = (float)(slot % 3 - 1), dy = (float)((slot / 3) % 3 - 1), dz = (float)(slot / 9 - 1);
                    for (int i = lo + lane; i < hi; i += 32) {
                        const float4 rec = xq_load(tv.xq, r0 + (i - o)), rl = xq_load(xl, r0 + (i - o));
                        float X, Y, Z, XL, YL, ZL;
                        shift_exact(rec.x, rl.x, dx, X, XL);
                        shift_exact(rec.y, rl.y, dy, Y, YL);
                        shift_exact(rec.z, rl.z, dz, Z, ZL);
                        list_store(buf, i - seg0, X, Y, Z, rec.w, XL, YL, ZL, rl.w);
                    }
                }
                if (lane == 0) {
                    if (own_pad && n_own >= seg0 && n_own < seg1) list_store_null(buf, n_own - seg0);
                    if (segn & 1) list_store_null(buf, segn);  // completes the last pair
                }
                __syncwarp();
                const int np = (segn + 1) >> 1, h = split ? (np + 1) >> 1 : np;
                const int pa = g ? h : 0, pe = g ? np : h;
                if constexpr (std::is_same<T, float>::value)
                    p2p_segment(buf, pa, pe, own_pairs - (seg0 >> 1), tx2, ty2, tz2, lx2, ly2, lz2, cs);
                else
                    p2p_segment_ff(buf, pa, pe, own_pairs - (seg0 >> 1), pt.x, pt.y, pt.z, pl.x, pl.y, pl.z, fs);
            }
            const double ih = tv.inv_h_leaf, ih2 = ih * ih;
            if constexpr (std::is_same<T, float>::value) {
                if (split) join_halves(cs);
                fphi = ((double)cs.ph + (double)cs.pl) * ih;
                fx = ((double)cs.xh + (double)cs.xl) * ih2;
                fy = ((double)cs.yh + (double)cs.yl) * ih2;
                fz = ((double)cs.zh + (double)cs.zl) * ih2;
            } else {
                ff sp = fs.p.get(), sx = fs.x.get(), sy = fs.y.get(), sz = fs.z.get();
                if (split) {  // the upper half-warp's sums join the lower one's
                    sp = ff_add(sp, ff_shfl_down(sp, 16));
                    sx = ff_add(sx, ff_shfl_down(sx, 16));
                    sy = ff_add(sy, ff_shfl_down(sy, 16));
                    sz = ff_add(sz, ff_shfl_down(sz, 16));
                }
                fphi = sp.to_double() * ih;
                fx = sx.to_double() * ih2;
                fy = sy.to_double() * ih2;
                fz = sz.to_double() * ih2;
            }
        }
        // far field from the leaf's local expansion
        if (Lrow) {
            T F, g0, g1, g2;
            T xs, ys, zs;
            if constexpr (sizeof(T) == 8) {
                xs = (T)((tv.x[tt] - cx) * tv.inv_h_leaf);
                ys = (T)((tv.y[tt] - cy) * tv.inv_h_leaf);
                zs = (T)((tv.z[tt] - cz) * tv.inv_h_leaf);
            } else {
                const float4 pt = xq_load(tv.xq, tt + r_own);
                xs = (T)pt.x; ys = (T)pt.y; zs = (T)pt.z;
            }
            if constexpr (sizeof(T) == 4) gen::GEN(l2p)<T>(SmemRowF{s_lrow[threadIdx.y]}, xs, ys, zs, F, g0, g1, g2);
            else if constexpr (std::is_same<T, ff>::value)
                gen::GEN(l2p)<T>(SmemRowFF{s_lrow_ff[threadIdx.y]}, xs, ys, zs, F, g0, g1, g2);
            else gen::GEN(l2p)<T>(RowLoad<T>{Lrow}, xs, ys, zs, F, g0, g1, g2);
            fphi += (double)F;
            fx -= (double)g0 * tv.inv_h_leaf;
            fy -= (double)g1 * tv.inv_h_leaf;
            fz -= (double)g2 * tv.inv_h_leaf;
        }
        if (valid && DAFMM_IN(tv.perm[t], tv.n, kChkPerm)) {
            const int o = tv.perm[t];
            if (phi) phi[o] = fphi;
            if (field) {
                field[3 * (size_t)o] = fx;
                field[3 * (size_t)o + 1] = fy;
                field[3 * (size_t)o + 2] = fz;
            }
        }
    }
}

// ---- adaptive trees ---------------------------------------------------------------------------
// Box geometry of an adaptive box (centre and width, precomputed per box at build time).
__device__ __forceinline__ void abox_geom(const AdaptiveView& av, int b, double& cx, double& cy, double& cz,
                                          double& h) {
    const double4 g = av.geom[b];
    cx = g.x;
    cy = g.y;
    cz = g.z;
    h = g.w;
}

__device__ __forceinline__ bool abox_is_leaf(const AdaptiveView& av, int b) {
    const int4 c0 = *reinterpret_cast<const int4*>(av.child + 8 * b);
    const int4 c1 = *reinterpret_cast<const int4*>(av.child + 8 * b + 4);
    return (c0.x & c0.y & c0.z & c0.w & c1.x & c1.y & c1.z & c1.w) < 0 &&
           c0.x < 0 && c0.y < 0 && c0.z < 0 && c0.w < 0 && c1.x < 0 && c1.y < 0 && c1.z < 0 && c1.w < 0;
}

// P2M (Eq. 2) at the leaves listed in `leaves`: one warp per leaf, as in k_p2m (H: the
// harmonic basis's free coefficients only, written at their layout positions)
template <class T, bool H = false>
__global__ void k_p2m_a(AdaptiveView av, const int* __restrict__ leaves, int nleaves, double* __restrict__ M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw) + threadIdx.y * (32 * 33);
    const int lane = threadIdx.x;
    const int li = blockIdx.x * blockDim.y + threadIdx.y;
    if (li >= nleaves) return;
    const int b = leaves[li];
    if (!DAFMM_IN(b, av.nbox, kChkBoxIndex)) return;
    double cx, cy, cz, h;
    abox_geom(av, b, cx, cy, cz, h);
    const double ih = 1.0 / h;
    int i0 = av.pbeg[b], i1 = av.pend[b];
    if (!DAFMM_RANGE(i0, i1, av.n, kChkBoxRange)) i0 = i1 = 0;
    if constexpr (sizeof(T) == 4) {  // the leaf's records
        if (!DAFMM_RANGE(av.xq0[b], (long long)av.xq0[b] + (i1 - i0), av.nrec, kChkRecord)) i0 = i1 = 0;
    }
    constexpr int NO = H ? nharm_of(P) : NC;
    constexpr int NJ = (NO + 31) / 32;
    T acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = T(0);
    ChunkSink<T, NJ, NO> sink{sm, lane, acc};
    for (int base = i0; base < i1; base += 32) {
        const int i = base + lane;
        T x = T(0), y = T(0), z = T(0), q = T(0);
        if (i < i1) {
            if constexpr (sizeof(T) == 4) {
                // the particle's FP32 record: its offset from this leaf's centre in leaf widths
                // (what the FP64 form computes, rounded once) and its charge, without FP64
                // instructions (1/64 of the FP32 rate on this part)
                const float4 r = xq_load(av.xq, av.xq0[b] + (i - i0));
                x = r.x;
                y = r.y;
                z = r.z;
                q = r.w;
            } else {
                x = (T)((av.x[i] - cx) * ih);
                y = (T)((av.y[i] - cy) * ih);
                z = (T)((av.z[i] - cz) * ih);
                q = (T)av.q[i];
            }
        }
        if constexpr (H) gen::GEN(p2mh)<T>(x, y, z, q, sink);
        else gen::GEN(p2m)<T>(x, y, z, q, sink);
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = lane + 32 * j;
        if (k < NO) M[(size_t)b * NCP + (H ? harm_full_index(k) : k)] = (double)acc[j];
    }
}

// M2M (Eq. 4) into the non-leaf boxes [lb, le) of one level, from their existing children
// (missing children count as zero; leaves keep their P2M result).  harm: harmonic multipoles,
// tab the harmonic M2M table -- free coefficients only, as in k_m2m.
template <class T>
__global__ void __launch_bounds__(256) k_m2m_a(ShiftTab tab, AdaptiveView av, int lb, int le, double* __restrict__ M,
                                               int harm) {
    constexpr int PP = m2m_parents<T>(), RS = 32 / PP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);  // [8][PP][NCP + 1]
    const int b0 = lb + blockIdx.x * PP;
    const int NO = harm ? nharm_of(P) : NC;
    for (int e = threadIdx.x; e < PP * NO; e += 256) {
        const int r = e / NO, j = e - r * NO;
        const int k = harm ? harm_full_index(j) : j;
        const int bx = b0 + r;
        T m[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int ch = bx < le ? av.child[8 * bx + c] : -1;
            m[c] = ch >= 0 && DAFMM_IN(ch, av.nbox, kChkBoxIndex) ? (T)M[(size_t)ch * NCP + k] : T(0);
        }
        hadamard8(m);
#pragma unroll
        for (int q = 0; q < 8; ++q) S[(q * PP + r) * (NCP + 1) + k] = m[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = lane % PP, sub = lane / PP;
    const int bx = b0 + r;
    if (bx >= le || abox_is_leaf(av, bx)) return;
    double* out = M + (size_t)bx * NCP;
    for (int j = w * RS + sub; j < NO; j += 8 * RS) {
        const int b = harm ? harm_full_index(j) : j;
        T acc = T(0);
        for (int e = tab.rowptr[b]; e < tab.rowptr[b + 1]; ++e)
            acc += tab_val<T>(tab, e) * S[(tab.par[e] * PP + r) * (NCP + 1) + tab.col[e]];
        out[b] = (double)acc;
    }
}

// M2L (Eq. 5) into the boxes tg[0..ntg) of one level that share the octant `oct`; the source
// of displacement v is child sc of the parent's colleague at offset a (c - v = 2a + sc)
template <class T, class Src>
__global__ void __launch_bounds__(256) k_m2l_a(const T* __restrict__ K, AdaptiveView av, const int* __restrict__ tg,
                                               const int* __restrict__ grp_ptr, int grp0, const Src* __restrict__ M,
                                               double* __restrict__ L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* src = reinterpret_cast<T*>(smem_raw);  // [32][NCP + 1]
    __shared__ int sidx[32];
    const int oct = blockIdx.y;
    int g0 = grp_ptr[grp0 + oct], g1 = grp_ptr[grp0 + oct + 1];
    if (!DAFMM_RANGE(g0, g1, av.nbox, kChkListPtr)) g0 = g1 = 0;
    const int t0 = g0 + blockIdx.x * 32;
    if (t0 >= g1) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ox = oct & 1, oy = (oct >> 1) & 1, oz = (oct >> 2) & 1;
    T acc[SH_ROWS];
#pragma unroll
    for (int j = 0; j < SH_ROWS; ++j) acc[j] = T(0);
    for (int vx = -3 + ox; vx <= 2 + ox; ++vx)
        for (int vy = -3 + oy; vy <= 2 + oy; ++vy)
            for (int vz = -3 + oz; vz <= 2 + oz; ++vz) {
                if (abs(vx) <= 1 && abs(vy) <= 1 && abs(vz) <= 1) continue;
                if (threadIdx.x < 32) {
                    const int ti = t0 + threadIdx.x;
                    int sbox = -1;
                    if (ti < g1 && DAFMM_IN(tg[ti], av.nbox, kChkBoxIndex) &&
                        DAFMM_IN(av.parent[tg[ti]], av.nbox, kChkBoxIndex)) {
                        const int P = av.parent[tg[ti]];
                        const int dx = ox - vx, dy = oy - vy, dz = oz - vz;  // = 2a + sc
                        const int scx = dx & 1, scy = dy & 1, scz = dz & 1;
                        const int ax = (dx - scx) >> 1, ay = (dy - scy) >> 1, az = (dz - scz) >> 1;
                        const int Q = av.colleague[27 * P + (ax + 1) * 9 + (ay + 1) * 3 + (az + 1)];
                        if (Q >= 0 && DAFMM_IN(Q, av.nbox, kChkBoxIndex))
                            sbox = av.child[8 * Q + (scx | (scy << 1) | (scz << 2))];
                        if (sbox >= 0 && !DAFMM_IN(sbox, av.nbox, kChkBoxIndex)) sbox = -1;
                    }
                    sidx[threadIdx.x] = sbox;
                }
                __syncthreads();
                for (int e = threadIdx.x; e < 32 * NC; e += 256) {
                    const int r = e / NC, k = e - r * NC;
                    const int sb = sidx[r];
                    src[r * (NCP + 1) + k] = sb >= 0 ? (T)M[(size_t)sb * NCP + k] : T(0);
                }
                __syncthreads();
                const int key = (vx + 3) * 49 + (vy + 3) * 7 + (vz + 3);
                const T* Kv = K + (size_t)key * NC * NCP;
                const T* srow = src + lane * (NCP + 1);
                const T* kw = Kv + (size_t)w * NCP;
#pragma unroll 1
                for (int a = 0; a < NC; ++a) {
                    const T sv = srow[a];
#pragma unroll
                    for (int j = 0; j < SH_ROWS; ++j)
                        if (w + 8 * j < NC) acc[j] = fma(kw[(size_t)(8 * j) * NCP + a], sv, acc[j]);
                }
                __syncthreads();
            }
    const int ti = t0 + lane;
    if (ti < g1 && DAFMM_IN(tg[ti], av.nbox, kChkBoxIndex)) {
        const int t = tg[ti];
        const double inv_h = 1.0 / av.geom[t].w;  // the target box's width (each tree has its own)
#pragma unroll
        for (int j = 0; j < SH_ROWS; ++j) {
            const int b = w + 8 * j;
            if (b < NC) L[(size_t)t * NCP + b] = (double)acc[j] * inv_h;
        }
    }
}

// P2L (Eq. 6): particles of the X-list leaves of each box of [lb, le) into its local expansion
template <class T>
__global__ void k_p2l_a(AdaptiveView av, int lb, int le, double* __restrict__ L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw) + threadIdx.y * (32 * 33);
    const int lane = threadIdx.x;
    const int b = lb + blockIdx.x * blockDim.y + threadIdx.y;
    if (b >= le) return;
    int x0i = av.x_ptr[b], x1i = av.x_ptr[b + 1];
    if (!DAFMM_RANGE(x0i, x1i, av.nx, kChkListPtr)) x0i = x1i = 0;
    if (x0i == x1i) return;
    double cx, cy, cz, h;
    abox_geom(av, b, cx, cy, cz, h);
    const double ih = 1.0 / h;
    constexpr int NJ = (NC + 31) / 32;
    T acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = T(0);
    ChunkSink<T, NJ> sink{sm, lane, acc};
    for (int xi = x0i; xi < x1i; ++xi) {
        const int c = av.x_idx[xi];
        if (!DAFMM_IN(c, av.nbox, kChkBoxIndex) || !DAFMM_RANGE(av.pbeg[c], av.pend[c], av.n, kChkBoxRange)) continue;
        const int i0 = av.pbeg[c], i1 = av.pend[c];
        for (int base = i0; base < i1; base += 32) {
            const int i = base + lane;
            T X = T(1), Y = T(0), Z = T(0), q = T(0);  // a dummy far point for idle lanes
            if (i < i1) {
                X = (T)((cx - av.x[i]) * ih);
                Y = (T)((cy - av.y[i]) * ih);
                Z = (T)((cz - av.z[i]) * ih);
                q = (T)av.q[i];
            }
            gen::GEN(p2l)<T>(X, Y, Z, q, sink);
        }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int k = lane + 32 * j;
        if (k < NC) L[(size_t)b * NCP + k] += (double)acc[j] * ih;
    }
}

// L2L (Eq. 7) from the parents [lb, le) of one level into their existing children (added to
// what M2L and P2L wrote)
template <class T>
__global__ void __launch_bounds__(256) k_l2l_a(ShiftTab tab, AdaptiveView av, int lb, int le, double* __restrict__ L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* src = reinterpret_cast<T*>(smem_raw);  // [32][NCP + 1]
    const int b0 = lb + blockIdx.x * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < 32 * NC; e += 256) {
        const int r = e / NC, k = e - r * NC;
        const int P = b0 + r;
        src[r * (NCP + 1) + k] = P < le ? (T)L[(size_t)P * NCP + k] : T(0);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 8) {
        // FP64 (bound by the FP64 pipe): lane = parent, every lane on the same row b
        const int P = b0 + lane;
        if (P >= le || abox_is_leaf(av, P)) return;
        int ch[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) ch[c] = av.child[8 * P + c];
        for (int b = w; b < NC; b += 8) {
            T R[8];
            l2l_row(tab, b, src + lane * (NCP + 1), R);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (ch[c] >= 0 && DAFMM_IN(ch[c], av.nbox, kChkBoxIndex)) L[(size_t)ch[c] * NCP + b] += (double)R[c];
        }
        return;
    }
    // FP32: warp w takes parents w, w + 8, ...; its lanes take consecutive rows b, so that the
    // read-modify-write of each child's row is one coalesced access per warp instead of 32
    // scattered ones (an ncu capture of the lane-per-parent form: long-scoreboard stalls 14 per
    // issue, the L2 hit rate 45 %; clustered N = 4e6, p = 10: L2L 3.69 -> 3.26 ms)
    for (int r = w; r < 32; r += 8) {
        const int P = b0 + r;
        if (P >= le || abox_is_leaf(av, P)) continue;
        int ch[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) ch[c] = av.child[8 * P + c];
        const T* srow = src + r * (NCP + 1);
        for (int b = lane; b < NC; b += 32) {
            T R[8];
            l2l_row(tab, b, srow, R);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (ch[c] >= 0 && DAFMM_IN(ch[c], av.nbox, kChkBoxIndex)) L[(size_t)ch[c] * NCP + b] += (double)R[c];
        }
    }
}

// leaves: P2P over the U list, M2P over the W list, L2P of the leaf's local expansion
template <class T>
__global__ void __launch_bounds__(256) k_leaf_a(AdaptiveView av, const int* __restrict__ leaves, int nleaves,
                                                const double* __restrict__ L, const double* __restrict__ M,
                                                const float* __restrict__ Mf, double* __restrict__ phi,
                                                double* __restrict__ field) {
    __shared__ float s_rows[8][2][NCP];  // per warp: the W box's multipoles and the leaf's locals, FP32
    extern __shared__ __align__(16) float4 s_list_a[];  // FP32: per warp kLeafSeg records (2 float4s each)
    const int lane = threadIdx.x;
    const int li = blockIdx.x * blockDim.y + threadIdx.y;
    if (li >= nleaves) return;
    float* mrow = s_rows[threadIdx.y][0];
    float* lrow = s_rows[threadIdx.y][1];
    const int b = leaves[li];
    if (!DAFMM_IN(b, av.nbox, kChkBoxIndex)) return;
    double cx, cy, cz, h;
    abox_geom(av, b, cx, cy, cz, h);
    const double ih = 1.0 / h;
    const int lev = av.level[b];
    if constexpr (sizeof(T) == 4) {
        if (lev >= 2) warp_row_to_f32(L + (size_t)b * NCP, lrow, lane);
    }
    int i0 = av.pbeg[b], i1 = av.pend[b];
    if (!DAFMM_RANGE(i0, i1, av.n, kChkBoxRange)) i0 = i1 = 0;
    if constexpr (sizeof(T) == 4) {  // the leaf's own records (its targets)
        if (!DAFMM_RANGE(av.xq0[b], (long long)av.xq0[b] + (i1 - i0), av.nrec, kChkRecord)) i0 = i1 = 0;
    }
    int u0 = av.u_ptr[b], u1 = av.u_ptr[b + 1];
    int w0 = av.w_ptr[b], w1 = av.w_ptr[b + 1];
    if (!DAFMM_RANGE(u0, u1, av.nu, kChkListPtr)) u0 = u1 = 0;
    if (!DAFMM_RANGE(w0, w1, av.nw, kChkListPtr)) w0 = w1 = 0;
    for (int base = i0; base < i1; base += 32) {
        // FP32: a pass of at most 16 targets splits the sources between the two half-warps,
        // lane l and lane l + 16 taking the same target
        const int m = min(32, i1 - base);
        const bool split = sizeof(T) == 4 && m <= 16;
        const int tl = split ? (lane & 15) : lane;
        const int t = base + tl;
        const bool valid = tl < m && (!split || lane < 16);  // the lanes that write
        const int tt = tl < m ? t : i0;
        double fphi = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        if constexpr (sizeof(T) == 8) {
            const double xt = av.x[tt], yt = av.y[tt], zt = av.z[tt];
            for (int ui = u0; ui < u1; ++ui) {
                const int sb = av.u_idx[ui];
                if (!DAFMM_IN(sb, av.nbox, kChkBoxIndex) || !DAFMM_RANGE(av.pbeg[sb], av.pend[sb], av.n, kChkBoxRange))
                    continue;
                for (int sidx = av.pbeg[sb]; sidx < av.pend[sb]; ++sidx) {
                    const double ex = xt - av.x[sidx], ey = yt - av.y[sidx], ez = zt - av.z[sidx];
                    const double r2 = ex * ex + ey * ey + ez * ez;
                    if (r2 > 0.0) {
                        const double ir = rsqrt(r2);
                        const double qr = av.q[sidx] * ir;
                        const double qr3 = qr * ir * ir;
                        fphi += qr;
                        fx += qr3 * ex; fy += qr3 * ey; fz += qr3 * ez;
                    }
                }
            }
        } else {
            const float4 pt = xq_load(av.xq, av.xq0[b] + (tt - i0)), pl = xq_load(av.xl, av.xq0[b] + (tt - i0));
            CompSums acc;  // in leaf widths of this leaf
            // The U-list leaves' records are copied into one shared-memory list in this leaf's
            // frame (source x h_s / h + centre offset / h, exactly: h_s / h is a power of two and
            // the rounding of the sum joins the remainder), the leaf's own records first, in
            // segments of up to kLeafSeg records; the pairwise sum runs over each segment.
            float4* buf = s_list_a + (size_t)threadIdx.y * 2 * kLeafSeg;
            const int g = split ? lane >> 4 : 0;
            const float2 tx2 = make_float2(pt.x, pt.x), ty2 = make_float2(pt.y, pt.y),
                         tz2 = make_float2(pt.z, pt.z);
            const float2 lx2 = make_float2(pl.x, pl.x), ly2 = make_float2(pl.y, pl.y),
                         lz2 = make_float2(pl.z, pl.z);
            int fill = 0, done = 0, own_end = 0;  // records in the segment, before it, of the own leaf
            auto flush = [&]() {
                if ((fill & 1) && lane == 0) list_store_null(buf, fill);  // completes the last pair
                __syncwarp();
                const int np = (fill + 1) >> 1, hp = split ? (np + 1) >> 1 : np;
                const int pa = g ? hp : 0, pe = g ? np : hp;
                p2p_segment(buf, pa, pe, (own_end - done) >> 1, tx2, ty2, tz2, lx2, ly2, lz2, acc);
                __syncwarp();  // the segment is no longer read
                done += fill;
                fill = 0;
            };
            const int* ijk_b = av.ijk + 3 * (size_t)b;
            auto add_leaf = [&](int sb) {
                // the source leaf's centre offset in this leaf's widths and its width ratio,
                // from the integer box coordinates (same tree): with d = lev_b - lev_s,
                // (c_s - c_b) / h_b = N / 2^(1 + max(0, -d)),
                // N = (2 i_s + 1) 2^max(0, d) - (2 i_b + 1) 2^max(0, -d) -- as hi + lo floats,
                // exactly, and without FP64 instructions (1/64 of the FP32 rate here)
                const int d = lev - av.level[sb];
                const int up = d > 0 ? d : 0, dn = d < 0 ? -d : 0;
                const float r = __int_as_float((127 + d) << 23);          // h_s / h_b = 2^d
                const float sc = __int_as_float((127 - 1 - dn) << 23);    // 2^-(1 + dn)
                const int* ijk_s = av.ijk + 3 * (size_t)sb;
                float oh[3], ol[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const long long N = ((2ll * ijk_s[k] + 1) << up) - ((2ll * ijk_b[k] + 1) << dn);
                    const float h = (float)N;
                    oh[k] = h * sc;
                    ol[k] = (float)(N - (long long)h) * sc;
                }
                const float ohx = oh[0], ohy = oh[1], ohz = oh[2];
                const float olx = ol[0], oly = ol[1], olz = ol[2];
                if (!DAFMM_RANGE(av.pbeg[sb], av.pend[sb], av.n, kChkBoxRange)) return;
                const int r0 = av.xq0[sb], n = av.pend[sb] - av.pbeg[sb];
                if (!DAFMM_RANGE(r0, (long long)r0 + n, av.nrec, kChkRecord)) return;
                for (int i0s = 0; i0s < n;) {
                    const int take = min(n - i0s, kLeafSeg - fill);
                    for (int i = lane; i < take; i += 32) {
                        const float4 rec = xq_load(av.xq, r0 + i0s + i), rl = xq_load(av.xl, r0 + i0s + i);
                        float X, Y, Z, XL, YL, ZL;
                        scale_shift_exact(rec.x, rl.x, r, ohx, olx, X, XL);
                        scale_shift_exact(rec.y, rl.y, r, ohy, oly, Y, YL);
                        scale_shift_exact(rec.z, rl.z, r, ohz, olz, Z, ZL);
                        list_store(buf, fill + i, X, Y, Z, rec.w, XL, YL, ZL, rl.w);
                    }
                    fill += take;
                    i0s += take;
                    if (fill == kLeafSeg) flush();
                }
            };
            // the leaf itself (the only records that can coincide with a target), completed to
            // an even count by a null record, then the other U-list leaves
            const int n_own = i1 - i0;
            own_end = n_own + (n_own & 1);  // (set first: a long own leaf flushes segments)
            add_leaf(b);
            if (n_own & 1) {
                if (lane == 0) list_store_null(buf, fill);  // fill < kLeafSeg here
                ++fill;
                if (fill == kLeafSeg) flush();
            }
            for (int ui = u0; ui < u1; ++ui) {
                const int sb = av.u_idx[ui];
                if (sb != b && DAFMM_IN(sb, av.nbox, kChkBoxIndex)) add_leaf(sb);
            }
            if (fill > 0) flush();
            if (split) join_halves(acc);
            fphi = ((double)acc.ph + (double)acc.pl) * ih;
            fx = ((double)acc.xh + (double)acc.xl) * ih * ih;
            fy = ((double)acc.yh + (double)acc.yl) * ih * ih;
            fz = ((double)acc.zh + (double)acc.zl) * ih * ih;
        }
        // M2P from the W list (Sec. 3.2): phi = F/h_w, E = -grad_s F / h_w^2
        if constexpr (sizeof(T) == 8) {
            for (int wi = w0; wi < w1; ++wi) {
                const int wb = av.w_idx[wi];
                if (!DAFMM_IN(wb, av.nbox, kChkBoxIndex)) continue;
                double wx, wy, wz, wh;
                abox_geom(av, wb, wx, wy, wz, wh);
                const double iwh = 1.0 / wh;
                T F, g0, g1, g2;
                const T sx0 = (T)((av.x[tt] - wx) * iwh), sy0 = (T)((av.y[tt] - wy) * iwh),
                        sz0 = (T)((av.z[tt] - wz) * iwh);
                gen::GEN(m2p)<T>(RowLoad<T>{M + (size_t)wb * NCP}, sx0, sy0, sz0, F, g0, g1, g2);
                fphi += (double)F * iwh;
                fx -= (double)g0 * iwh * iwh;
                fy -= (double)g1 * iwh * iwh;
                fz -= (double)g2 * iwh * iwh;
            }
        } else {
            // FP32, without FP64 instructions (this part runs FP64 at 1/64 of the FP32 rate): the
            // W box is finer than the leaf by dl levels of the same tree, so with integer box
            // coordinates i at each level (c_b - c_w) / h_w = ((2 i_b + 1) 2^dl - (2 i_w + 1)) / 2
            // per axis, exactly; the target in the W box's frame is its leaf-frame offset (record
            // and remainder) times 2^dl plus that; the box's multipoles come as FP32 rows (Mf).
            // Its terms are summed in FP32 and join the FP64 sums once per target.
            const float4 pw = xq_load(av.xq, av.xq0[b] + (tt - i0)), plw = xq_load(av.xl, av.xq0[b] + (tt - i0));
            const float ihf = (float)ih;
            float wphi = 0.f, wfx = 0.f, wfy = 0.f, wfz = 0.f;
            const int* ib = av.ijk + 3 * (size_t)b;
            for (int wi = w0; wi < w1; ++wi) {
                const int wb = av.w_idx[wi];
                if (!DAFMM_IN(wb, av.nbox, kChkBoxIndex)) continue;
                const int dl = av.level[wb] - lev;
                float sx0, sy0, sz0, iw;
                if (dl >= 0 && dl <= 30) {
                    const float r = (float)(1u << dl);
                    const long long rr = 1ll << dl;
                    const int* iwb = av.ijk + 3 * (size_t)wb;
                    const float ox = 0.5f * (float)((2ll * ib[0] + 1) * rr - (2ll * iwb[0] + 1));
                    const float oy = 0.5f * (float)((2ll * ib[1] + 1) * rr - (2ll * iwb[1] + 1));
                    const float oz = 0.5f * (float)((2ll * ib[2] + 1) * rr - (2ll * iwb[2] + 1));
                    sx0 = fmaf(plw.x, r, fmaf(pw.x, r, ox));
                    sy0 = fmaf(plw.y, r, fmaf(pw.y, r, oy));
                    sz0 = fmaf(plw.z, r, fmaf(pw.z, r, oz));
                    iw = ihf * r;
                } else {  // (not a W-list shape; kept general)
                    double wx, wy, wz, wh;
                    abox_geom(av, wb, wx, wy, wz, wh);
                    const double iwh = 1.0 / wh;
                    sx0 = (float)((av.x[tt] - wx) * iwh);
                    sy0 = (float)((av.y[tt] - wy) * iwh);
                    sz0 = (float)((av.z[tt] - wz) * iwh);
                    iw = (float)iwh;
                }
                if (Mf) warp_row_f32(Mf + (size_t)wb * NCP, mrow, lane);
                else warp_row_to_f32(M + (size_t)wb * NCP, mrow, lane);
                T F, g0, g1, g2;
                gen::GEN(m2p)<T>(SmemRowF{mrow}, sx0, sy0, sz0, F, g0, g1, g2);
                wphi = fmaf(F, iw, wphi);
                const float iw2 = iw * iw;
                wfx = fmaf(-g0, iw2, wfx);
                wfy = fmaf(-g1, iw2, wfy);
                wfz = fmaf(-g2, iw2, wfz);
            }
            fphi += (double)wphi;
            fx += (double)wfx;
            fy += (double)wfy;
            fz += (double)wfz;
        }
        // L2P of this leaf's local expansion
        if (lev >= 2) {
            T F, g0, g1, g2;
            T xs, ys, zs;
            if constexpr (sizeof(T) == 8) {
                xs = (T)((av.x[tt] - cx) * ih);
                ys = (T)((av.y[tt] - cy) * ih);
                zs = (T)((av.z[tt] - cz) * ih);
            } else {
                const float4 pt = xq_load(av.xq, av.xq0[b] + (tt - i0));
                xs = (T)pt.x; ys = (T)pt.y; zs = (T)pt.z;
            }
            if constexpr (sizeof(T) == 4) gen::GEN(l2p)<T>(SmemRowF{lrow}, xs, ys, zs, F, g0, g1, g2);
            else gen::GEN(l2p)<T>(RowLoad<T>{L + (size_t)b * NCP}, xs, ys, zs, F, g0, g1, g2);
            fphi += (double)F;
            fx -= (double)g0 * ih;
            fy -= (double)g1 * ih;
            fz -= (double)g2 * ih;
        }
        if (valid && DAFMM_IN(av.perm[t], av.n, kChkPerm)) {
            const int o = av.perm[t];
            if (phi) phi[o] = fphi;
            if (field) {
                field[3 * (size_t)o] = fx;
                field[3 * (size_t)o + 1] = fy;
                field[3 * (size_t)o + 2] = fz;
            }
        }
    }
}

// ---- single-operator batches ------------------------------------------------------------------
template <class T>
struct RowStore {
    double* o;
    __device__ __forceinline__ void operator()(int k, T v) const { o[k] = (double)v; }
};

template <class T>
__global__ void k_op_p2m(int64_t n, const double* __restrict__ s, const double* __restrict__ q, double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    gen::GEN(p2m)<T>((T)s[3 * i], (T)s[3 * i + 1], (T)s[3 * i + 2], (T)q[i], RowStore<T>{out + i * NC});
}
template <class T>
__global__ void k_op_p2l(int64_t n, const double* __restrict__ w, const double* __restrict__ q, double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    gen::GEN(p2l)<T>((T)w[3 * i], (T)w[3 * i + 1], (T)w[3 * i + 2], (T)q[i], RowStore<T>{out + i * NC});
}
template <class T, bool M2P>
__global__ void k_op_eval(int64_t n, const double* __restrict__ C, const double* __restrict__ x, double* out4) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T F, g0, g1, g2;
    if (M2P) gen::GEN(m2p)<T>(RowLoad<T>{C + i * NC}, (T)x[3 * i], (T)x[3 * i + 1], (T)x[3 * i + 2], F, g0, g1, g2);
    else gen::GEN(l2p)<T>(RowLoad<T>{C + i * NC}, (T)x[3 * i], (T)x[3 * i + 1], (T)x[3 * i + 2], F, g0, g1, g2);
    out4[4 * i] = (double)F;
    out4[4 * i + 1] = (double)g0;
    out4[4 * i + 2] = (double)g1;
    out4[4 * i + 3] = (double)g2;
}
template <class T>
__global__ void k_op_shift(ShiftTab tab, int64_t n, const int* __restrict__ oct, const double* __restrict__ in,
                           double* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = oct[i] & 7;
    for (int b = 0; b < NC; ++b) {
        T s = T(0);
        for (int e = tab.rowptr[b]; e < tab.rowptr[b + 1]; ++e) {
            T v = tab_val<T>(tab, e);
            if (__popc(tab.par[e] & c) & 1) v = -v;
            s += v * (T)in[i * NC + tab.col[e]];
        }
        out[i * NC + b] = (double)s;
    }
}

// ---- launchers ---------------------------------------------------------------------------------
template <class K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

static cudaError_t p2m_launch(const TreeView& tv, int prec, double* M, const F16Rows* f16, cudaStream_t s) {
    if (tv.nleaf == 0) return cudaSuccess;
    const F16Rows fr = f16 ? *f16 : F16Rows{};
    const int rows32 = (prec & kRowsF32) ? 1 : 0;
    const bool harm = (prec & kRowsHarm) != 0;
    prec &= ~(kRowsF32 | kRowsHarm);
    const bool f64 = prec == DAFMM_FP64, fff = prec == DAFMM_FF;
    if (harm && (f64 || fff)) return cudaErrorInvalidValue;  // (the FP32 kernel only)
    // the fused F16 split: FP32 harmonic rows, every padded row position held by the warp
    if (fr.hi && (!harm || !rows32 || !fr.lo || !fr.inv || fr.rowlen < nharm_of(P) ||
                  fr.rowlen > 32 * ((nharm_of(P) + 31) / 32)))
        return cudaErrorInvalidValue;
    const size_t per_warp = (size_t)32 * 33 * (f64 || fff ? 8 : 4);
    int wpb = (int)((96 * 1024) / per_warp);
    wpb = wpb < 1 ? 1 : (wpb > 4 ? 4 : wpb);
    const size_t smem = per_warp * wpb;
    dim3 blk(32, wpb), grd((tv.nleaf + wpb - 1) / wpb);
    cudaError_t e;
    if (f64) {
        if ((e = set_smem(k_p2m<double>, smem)) != cudaSuccess) return e;
        k_p2m<double><<<grd, blk, smem, s>>>(tv, M, 0, F16Rows{});
    } else if (fff) {
        if ((e = set_smem(k_p2m<ff>, smem)) != cudaSuccess) return e;
        k_p2m<ff><<<grd, blk, smem, s>>>(tv, M, 0, F16Rows{});
    } else if (harm) {
        if ((e = set_smem(k_p2m<float, true>, smem)) != cudaSuccess) return e;
        k_p2m<float, true><<<grd, blk, smem, s>>>(tv, M, rows32, fr);
    } else {
        if ((e = set_smem(k_p2m<float>, smem)) != cudaSuccess) return e;
        k_p2m<float><<<grd, blk, smem, s>>>(tv, M, rows32, F16Rows{});
    }
    return cudaGetLastError();
}

static cudaError_t m2m_launch(const OrderData& od, int prec, int lc, const double* Mc, double* Mp,
                              cudaStream_t s) {
    const int rows32 = (prec & kRowsF32) ? 1 : 0;
    const int harm = (prec & kRowsHarm) ? 1 : 0;
    prec &= ~(kRowsF32 | kRowsHarm);
    if (harm && (prec == DAFMM_FP64 || prec == DAFMM_FF || !od.m2mh_rowptr)) return cudaErrorInvalidValue;
    const int Pc = 1 << (lc - 1);
    const int nparent = Pc * Pc * Pc;
    const bool f32 = prec == DAFMM_FP32;
    const ShiftTab tab = harm ? od.m2mh() : od.m2m();
    cudaError_t e;
    if (!f32) {
        constexpr int PP = m2m_parents<double>();
        if ((e = set_smem(k_m2m<double>, m2m_smem<double>())) != cudaSuccess) return e;
        k_m2m<double><<<(nparent + PP - 1) / PP, 256, m2m_smem<double>(), s>>>(tab, lc, Mc, Mp, 0, harm);
    } else {
        constexpr int PP = m2m_parents<float>();
        if ((e = set_smem(k_m2m<float>, m2m_smem<float>())) != cudaSuccess) return e;
        k_m2m<float><<<(nparent + PP - 1) / PP, 256, m2m_smem<float>(), s>>>(tab, lc, Mc, Mp, rows32, harm);
    }
    return cudaGetLastError();
}

static cudaError_t l2l_launch(const OrderData& od, int prec, int lc, const double* Lp, double* Lc,
                              cudaStream_t s) {
    const int Pc = 1 << (lc - 1);
    const int nparent = Pc * Pc * Pc;
    const bool f32 = prec == DAFMM_FP32;
    const size_t smem = (size_t)32 * (NCP + 1) * (f32 ? 4 : 8);
    cudaError_t e;
    dim3 grd((nparent + 31) / 32);
    if (!f32) {
        if ((e = set_smem(k_l2l<double>, smem)) != cudaSuccess) return e;
        k_l2l<double><<<grd, 256, smem, s>>>(od.l2l(), lc, Lp, Lc);
    } else {
        if ((e = set_smem(k_l2l<float>, smem)) != cudaSuccess) return e;
        k_l2l<float><<<grd, 256, smem, s>>>(od.l2l(), lc, Lp, Lc);
    }
    return cudaGetLastError();
}

static cudaError_t m2l_launch(const OrderData& od, int prec, int l, const double* M, const float* Mf,
                              double* L, double inv_h, cudaStream_t s) {
    const int Pp = 1 << (l - 1);
    const int nlin = Pp * Pp * Pp;
    dim3 grd((nlin + 31) / 32, 8);
    cudaError_t e;
    if (prec == DAFMM_FP64) {
        const size_t smem = (size_t)32 * (NCP + 1) * 8;
        if ((e = set_smem(k_m2l<double, double>, smem)) != cudaSuccess) return e;
        k_m2l<double, double><<<grd, 256, smem, s>>>(od.K64, l, M, L, inv_h);
    } else {
        const size_t smem = (size_t)32 * (NCP + 1) * 4;
        if ((e = set_smem(k_m2l<float, float>, smem)) != cudaSuccess) return e;
        k_m2l<float, float><<<grd, 256, smem, s>>>(od.K32, l, Mf, L, inv_h);
    }
    return cudaGetLastError();
}

static cudaError_t leaf_launch(const TreeView& tv, int prec, const double* Lleaf, double* phi, double* field,
                               cudaStream_t s) {
    if (tv.nleaf == 0) return cudaSuccess;
    dim3 blk(32, 4), grd((tv.nleaf + 3) / 4);
    if (prec == DAFMM_FP64) k_leaf<double><<<grd, blk, 0, s>>>(tv, Lleaf, phi, field);
    else if (prec == DAFMM_FF) k_leaf<ff><<<grd, blk, 0, s>>>(tv, Lleaf, phi, field);
    else k_leaf<float><<<grd, blk, 0, s>>>(tv, Lleaf, phi, field);
    return cudaGetLastError();
}

// M2L by rotation at level l (FP64, uniform trees): L~ = (1/h) sum_v B_v A_|v| F_v M~
// the task lists and expansion steps of the rotation: harmonic (free outputs only) or full
static RotLists rot_lists(const OrderData& od, bool harm) {
    if (harm) return RotLists{od.rot_lxh, od.rot_lzh, od.rot_lah, od.rot_lenh[0], od.rot_lenh[1], od.rot_lenh[2]};
    return RotLists{od.rot_lx, od.rot_lz, od.rot_la, od.rot_len[0], od.rot_len[1], od.rot_len[2]};
}
static RotHarm rot_harm(const OrderData& od) {
    RotHarm hm;
    hm.step = od.hxr_step;
    hm.w = od.hxr_w;
    for (int k = 0; k < kMaxOrder + 3; ++k) hm.cst[k] = od.hxr_cst[k];
    return hm;
}

static cudaError_t m2l_rot_launch(const OrderData& od, int l, const double* M, double* L, double inv_h, bool harm,
                                  cudaStream_t s) {
    const int nbox = 1 << (3 * l);
    harm = harm && od.rot_lxh;
    const RotLists rl = rot_lists(od, harm);
    const RotHarm hm = rot_harm(od);
    if (harm)
        k_m2l_rot<double, true><<<(nbox + 7) / 8, 256, 0, s>>>(od.rot_T, od.rot_rho, rl, od.ax_val, od.ax_nnz, l, M,
                                                                nullptr, nullptr, L, inv_h, hm);
    else
        k_m2l_rot<double, false><<<(nbox + 7) / 8, 256, 0, s>>>(od.rot_T, od.rot_rho, rl, od.ax_val, od.ax_nnz, l, M,
                                                                 nullptr, nullptr, L, inv_h, hm);
    return cudaGetLastError();
}

// the same in float-float (DAFMM_FF): tables od.rot_Tf, od.ax_valf; the source rows' FP32 parts
// Mh, Ml (k_split_ff); the task lists staged in shared memory
static cudaError_t m2l_rot_ff_launch(const OrderData& od, int l, const float* Mh, const float* Ml, double* L,
                                     double inv_h, bool harm, cudaStream_t s) {
    const int nbox = 1 << (3 * l);
    harm = harm && od.rot_lxh;
    const RotLists rl = rot_lists(od, harm);
    const RotHarm hm = rot_harm(od);
    const ff* T = reinterpret_cast<const ff*>(od.rot_Tf);
    const ff* av = reinterpret_cast<const ff*>(od.ax_valf);
    if (harm)
        k_m2l_rot<ff, true><<<(nbox + 7) / 8, 256, 0, s>>>(T, od.rot_rho, rl, av, od.ax_nnz, l, nullptr, Mh, Ml, L,
                                                            inv_h, hm);
    else
        k_m2l_rot<ff, false><<<(nbox + 7) / 8, 256, 0, s>>>(T, od.rot_rho, rl, av, od.ax_nnz, l, nullptr, Mh, Ml, L,
                                                             inv_h, hm);
    return cudaGetLastError();
}

static cudaError_t split_ff_launch(const double* a, float* hi, float* lo, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = (n + 255) / 256;
    k_split_ff<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(a, hi, lo, n);
    return cudaGetLastError();
}

static cudaError_t to_ff_launch(const double* a, float2* b, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t blocks = (n + 255) / 256;
    k_to_ff<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(a, reinterpret_cast<ff*>(b), n);
    return cudaGetLastError();
}

// the rotation tables of all keys and the axial matrices of the nrho lengths in r0s (3 per
// length, along x); Kscratch holds nrho dense matrices
static cudaError_t rot_setup_launch(OrderData& od, const double* r0s, int nrho, double* Kscratch, cudaStream_t s) {
    k_kgen<<<nrho, 256, 0, s>>>(od.mul(), Kscratch, nullptr, -1, nullptr, r0s);
    k_axial_gather<<<nrho, 256, 0, s>>>(Kscratch, od.ax_rowptr, od.ax_col, od.ax_nnz, od.ax_val);
    k_rot_tables<<<kNumKeys, 128, 0, s>>>(od.rot_T);
    return cudaGetLastError();
}

// the matrices of the given keys (all keys when key_list is null)
static cudaError_t kgen_launch(OrderData& od, const short* key_list, int nkeys, cudaStream_t s) {
    if (nkeys <= 0) return cudaSuccess;
    k_kgen<<<key_list ? nkeys : kNumKeys, 256, 0, s>>>(od.mul(), od.K64, od.K32, -1, key_list, nullptr);
    return cudaGetLastError();
}

// ---- adaptive launchers ----
static cudaError_t p2m_a_launch(const AdaptiveView& av, const int* leaves, int nleaves, int prec, double* M,
                                cudaStream_t s) {
    if (nleaves == 0) return cudaSuccess;
    const bool harm = (prec & kRowsHarm) != 0;
    prec &= ~kRowsHarm;
    const bool f64 = prec == DAFMM_FP64;
    if (harm && (f64 || prec == DAFMM_FF)) return cudaErrorInvalidValue;  // (the FP32 kernel only)
    const size_t per_warp = (size_t)32 * 33 * (f64 ? 8 : 4);
    int wpb = (int)((96 * 1024) / per_warp);
    wpb = wpb < 1 ? 1 : (wpb > 4 ? 4 : wpb);
    const size_t smem = per_warp * wpb;
    dim3 blk(32, wpb), grd((nleaves + wpb - 1) / wpb);
    cudaError_t e;
    if (f64) {
        if ((e = set_smem(k_p2m_a<double>, smem)) != cudaSuccess) return e;
        k_p2m_a<double><<<grd, blk, smem, s>>>(av, leaves, nleaves, M);
    } else if (harm) {
        if ((e = set_smem(k_p2m_a<float, true>, smem)) != cudaSuccess) return e;
        k_p2m_a<float, true><<<grd, blk, smem, s>>>(av, leaves, nleaves, M);
    } else {
        if ((e = set_smem(k_p2m_a<float>, smem)) != cudaSuccess) return e;
        k_p2m_a<float><<<grd, blk, smem, s>>>(av, leaves, nleaves, M);
    }
    return cudaGetLastError();
}

static cudaError_t m2m_a_launch(const OrderData& od, const AdaptiveView& av, int prec, int lb, int le, double* M,
                                cudaStream_t s) {
    if (le <= lb) return cudaSuccess;
    const int harm = (prec & kRowsHarm) ? 1 : 0;
    prec &= ~kRowsHarm;
    if (harm && (prec == DAFMM_FP64 || prec == DAFMM_FF || !od.m2mh_rowptr)) return cudaErrorInvalidValue;
    const bool f32 = prec == DAFMM_FP32;
    const ShiftTab tab = harm ? od.m2mh() : od.m2m();
    cudaError_t e;
    if (!f32) {
        constexpr int PP = m2m_parents<double>();
        if ((e = set_smem(k_m2m_a<double>, m2m_smem<double>())) != cudaSuccess) return e;
        k_m2m_a<double><<<(le - lb + PP - 1) / PP, 256, m2m_smem<double>(), s>>>(tab, av, lb, le, M, harm);
    } else {
        constexpr int PP = m2m_parents<float>();
        if ((e = set_smem(k_m2m_a<float>, m2m_smem<float>())) != cudaSuccess) return e;
        k_m2m_a<float><<<(le - lb + PP - 1) / PP, 256, m2m_smem<float>(), s>>>(tab, av, lb, le, M, harm);
    }
    return cudaGetLastError();
}

static cudaError_t m2l_a_launch(const OrderData& od, const AdaptiveView& av, int prec, const int* tg,
                                const int* grp_ptr, int grp0, int max_group, const double* M, const float* Mf,
                                double* L, cudaStream_t s) {
    if (max_group == 0) return cudaSuccess;
    if (prec & kM2LRot) {  // FP64 by rotation (Sec. 3.4)
        const bool harm = (prec & kM2LHarm) && od.rot_lxh;
        const RotLists rl = rot_lists(od, harm);
        const RotHarm hm = rot_harm(od);
        const dim3 grd((max_group + 7) / 8, 8);
        if (harm)
            k_m2l_rot_a<true><<<grd, 256, 0, s>>>(od.rot_T, od.rot_rho, rl, od.ax_val, od.ax_nnz, av, tg, grp_ptr, grp0,
                                                  M, L, hm);
        else
            k_m2l_rot_a<false><<<grd, 256, 0, s>>>(od.rot_T, od.rot_rho, rl, od.ax_val, od.ax_nnz, av, tg, grp_ptr,
                                                   grp0, M, L, hm);
        return cudaGetLastError();
    }
    dim3 grd((max_group + 31) / 32, 8);
    cudaError_t e;
    if (prec == DAFMM_FP64) {
        const size_t smem = (size_t)32 * (NCP + 1) * 8;
        if ((e = set_smem(k_m2l_a<double, double>, smem)) != cudaSuccess) return e;
        k_m2l_a<double, double><<<grd, 256, smem, s>>>(od.K64, av, tg, grp_ptr, grp0, M, L);
    } else {
        const size_t smem = (size_t)32 * (NCP + 1) * 4;
        if ((e = set_smem(k_m2l_a<float, float>, smem)) != cudaSuccess) return e;
        k_m2l_a<float, float><<<grd, 256, smem, s>>>(od.K32, av, tg, grp_ptr, grp0, Mf, L);
    }
    return cudaGetLastError();
}

static cudaError_t p2l_a_launch(const AdaptiveView& av, int prec, int lb, int le, double* L, cudaStream_t s) {
    if (le <= lb) return cudaSuccess;
    const bool f64 = prec == DAFMM_FP64;
    const size_t per_warp = (size_t)32 * 33 * (f64 ? 8 : 4);
    int wpb = (int)((96 * 1024) / per_warp);
    wpb = wpb < 1 ? 1 : (wpb > 4 ? 4 : wpb);
    const size_t smem = per_warp * wpb;
    dim3 blk(32, wpb), grd((le - lb + wpb - 1) / wpb);
    cudaError_t e;
    if (f64) {
        if ((e = set_smem(k_p2l_a<double>, smem)) != cudaSuccess) return e;
        k_p2l_a<double><<<grd, blk, smem, s>>>(av, lb, le, L);
    } else {
        if ((e = set_smem(k_p2l_a<float>, smem)) != cudaSuccess) return e;
        k_p2l_a<float><<<grd, blk, smem, s>>>(av, lb, le, L);
    }
    return cudaGetLastError();
}

static cudaError_t l2l_a_launch(const OrderData& od, const AdaptiveView& av, int prec, int lb, int le, double* L,
                                cudaStream_t s) {
    if (le <= lb) return cudaSuccess;
    const bool f32 = prec == DAFMM_FP32;
    const size_t smem = (size_t)32 * (NCP + 1) * (f32 ? 4 : 8);
    dim3 grd((le - lb + 31) / 32);
    cudaError_t e;
    if (!f32) {
        if ((e = set_smem(k_l2l_a<double>, smem)) != cudaSuccess) return e;
        k_l2l_a<double><<<grd, 256, smem, s>>>(od.l2l(), av, lb, le, L);
    } else {
        if ((e = set_smem(k_l2l_a<float>, smem)) != cudaSuccess) return e;
        k_l2l_a<float><<<grd, 256, smem, s>>>(od.l2l(), av, lb, le, L);
    }
    return cudaGetLastError();
}

static cudaError_t leaf_a_launch(const AdaptiveView& av, const int* leaves, int nleaves, int prec, const double* L,
                                 const double* M, const float* Mf, double* phi, double* field, int warps,
                                 cudaStream_t s) {
    if (nleaves == 0) return cudaSuccess;
    warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
    dim3 blk(32, warps), grd((nleaves + warps - 1) / warps);
    if (prec == DAFMM_FP64) {
        k_leaf_a<double><<<grd, blk, 0, s>>>(av, leaves, nleaves, L, M, nullptr, phi, field);
    } else {
        const size_t smem = (size_t)warps * 2 * kLeafSeg * sizeof(float4);
        cudaError_t e = cudaFuncSetAttribute(k_leaf_a<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_leaf_a<float><<<grd, blk, smem, s>>>(av, leaves, nleaves, L, M, Mf, phi, field);
    }
    return cudaGetLastError();
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 127) / 128); }

static cudaError_t op_p2m(int prec, int64_t n, const double* sv, const double* q, double* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == DAFMM_FP64) k_op_p2m<double><<<nblk(n), 128, 0, s>>>(n, sv, q, out);
    else k_op_p2m<float><<<nblk(n), 128, 0, s>>>(n, sv, q, out);
    return cudaGetLastError();
}
static cudaError_t op_p2l(int prec, int64_t n, const double* w, const double* q, double* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == DAFMM_FP64) k_op_p2l<double><<<nblk(n), 128, 0, s>>>(n, w, q, out);
    else k_op_p2l<float><<<nblk(n), 128, 0, s>>>(n, w, q, out);
    return cudaGetLastError();
}
static cudaError_t op_l2p(int prec, int64_t n, const double* L, const double* x, double* out4, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == DAFMM_FP64) k_op_eval<double, false><<<nblk(n), 128, 0, s>>>(n, L, x, out4);
    else k_op_eval<float, false><<<nblk(n), 128, 0, s>>>(n, L, x, out4);
    return cudaGetLastError();
}
static cudaError_t op_m2p(int prec, int64_t n, const double* M, const double* x, double* out4, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == DAFMM_FP64) k_op_eval<double, true><<<nblk(n), 128, 0, s>>>(n, M, x, out4);
    else k_op_eval<float, true><<<nblk(n), 128, 0, s>>>(n, M, x, out4);
    return cudaGetLastError();
}
static cudaError_t op_shift(const OrderData& od, int which, int prec, int64_t n, const int* oct,
                            const double* in, double* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const ShiftTab t = which == 0 ? od.m2m() : od.l2l();
    if (prec == DAFMM_FP64) k_op_shift<double><<<nblk(n), 128, 0, s>>>(t, n, oct, in, out);
    else k_op_shift<float><<<nblk(n), 128, 0, s>>>(t, n, oct, in, out);
    return cudaGetLastError();
}

}  // namespace ord_P

const OrderOps* DAFMM_CAT(order_ops_p, DAFMM_P)() {
    using namespace DAFMM_CAT(ord_, DAFMM_P);
    static const OrderOps ops = {
        P, NC, NCP,
        HostShiftTable{gen::GENT(m2m, _nnz), gen::GENT(m2m, _rowptr), gen::GENT(m2m, _col), gen::GENT(m2m, _par),
                       gen::GENT(m2m, _val)},
        HostShiftTable{gen::GENT(l2l, _nnz), gen::GENT(l2l, _rowptr), gen::GENT(l2l, _col), gen::GENT(l2l, _par),
                       gen::GENT(l2l, _val)},
        HostShiftTable{gen::GENT(m2mh, _nnz), gen::GENT(m2mh, _rowptr), gen::GENT(m2mh, _col), gen::GENT(m2mh, _par),
                       gen::GENT(m2mh, _val)},
        p2m_launch, m2m_launch, l2l_launch, m2l_launch, leaf_launch, kgen_launch, m2l_rot_launch, rot_setup_launch,
        ROT_TSZ,
        op_p2m, op_p2l, op_l2p, op_m2p, op_shift,
        p2m_a_launch, m2m_a_launch, m2l_a_launch, p2l_a_launch, l2l_a_launch, leaf_a_launch,
        m2l_rot_ff_launch, to_ff_launch, split_ff_launch};
    return &ops;
}

}  // namespace dafmm
