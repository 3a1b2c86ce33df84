// tc_common.cuh -- pieces shared by the tensor-core contraction kernels (tc_ops.cu: operands
// by TMA boxes; tc_gather.cu: source rows gathered per target): PTX wrappers for mbarriers,
// TMA, tcgen05 MMA / TMEM, the per-order tile configuration, the term sequence of a work
// item, the TF32 split, and the host-side tensor-map encoding.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_ops.h"

namespace dafmm {
namespace tc {

// ---- PTX wrappers ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr long long kWaitLimit = 1ll << 24;  // try_wait rounds before a wait is declared stuck

// bounded wait; on expiry records `code` in *err and returns false
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    atomicExch(err, code);
    return false;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);        // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                         // swizzle mode: 128-byte
    return d;
}

// instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                      // D format F32
           | (2u << 7) | (2u << 10)       // A, B format TF32
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// instruction descriptor of kind::f16 with both operands F16: D = F32, A = B = F16, K-major
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4)                      // D format F32
           | (0u << 7) | (0u << 10)       // A, B format F16
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// one MMA step of the split product with TF32 (H = false) or F16 (H = true) operands
template <bool H>
__device__ __forceinline__ void mma_op(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (H) mma_f16(dtmem, adesc, bdesc, idesc, acc);
    else mma_tf32(dtmem, adesc, bdesc, idesc, acc);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// TMEM loads: the load and tcgen05.wait::ld sit in one asm statement, so the outputs are
// defined only after the wait and no use of a register can be scheduled before it landed.
// 32 lanes x 16 columns, load and wait in one statement
__device__ __forceinline__ void tmem_ld16w(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}


// ---- configuration per order ------------------------------------------------------------------
// H = false: TF32 operands (rows of ncp FP32 values); H = true: F16 operands (rows of ncph =
// ncoef rounded up to 16 halves).  Either way a K chunk is 128 bytes of a row (32 TF32 or 64
// F16 values) and one MMA step takes 32 bytes of it (K = 8 or 16).
template <int P, bool H = false>
struct Cfg {
    static constexpr int NC = ncoef_of(P);
    static constexpr int NCP = ncp_of(P);
    static constexpr int ROWLEN = H ? (NC + 15) / 16 * 16 : NCP;  // operand row length, elements
    static constexpr int KPC = H ? 64 : 32;                         // elements per 128-byte chunk
    static constexpr int KSTEP = H ? 16 : 8;                        // elements per MMA step
    static constexpr int NPF = (NC + 15) / 16 * 16;               // N padded to the MMA granule
    static constexpr int NHALF = NPF > 192 ? 2 : 1;                // N split: <= 192 register sums per thread
    static constexpr int NP = NHALF == 1 ? NPF : (NPF / 2 + 15) / 16 * 16;
    static constexpr int NKC = (ROWLEN + KPC - 1) / KPC;           // K chunks of 128 bytes
    static constexpr int KSTEPS_LAST = (ROWLEN - KPC * (NKC - 1)) / KSTEP;  // MMA steps in the last chunk
    static constexpr int A_BYTES = 128 * 128;
    // B rows loaded per stage: the coefficients rounded up to 8 (one swizzle atom).  The MMA
    // reads NP >= NPL rows; rows NPL..NP-1 belong to whatever follows in shared memory and only
    // reach accumulator columns that are never used (columns of D depend on rows of B alone).
    // At p = 8 this saves the stage bytes that make room for a third pipeline stage.
    static constexpr int NPL = NHALF == 1 ? (NC + 7) / 8 * 8 : NP;
    static constexpr int B_BYTES = NPL * 128;
    static constexpr int SLACK = (NP - NPL) * 128;  // over-read past the last stage stays in the block
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int SMEM_AVAIL = 227 * 1024 - 2048 - SLACK;
    static constexpr int STAGES = (SMEM_AVAIL / STAGE_BYTES) > 4 ? 4 : (SMEM_AVAIL / STAGE_BYTES);
    static constexpr int TMEM_COLS = 2 * NP <= 256 ? 256 : 512;
    static constexpr uint32_t IDESC = H ? idesc_f16(128, NP) : idesc_tf32(128, NP);
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + SLACK + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(NPL <= NP && NPL >= NC - (NHALF - 1) * NP, "loaded B rows");
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= 192, "MMA N");
    static_assert(STAGES >= 2, "pipeline depth");
    static_assert(2 * NP <= TMEM_COLS, "TMEM double buffer");
    static_assert(ROWLEN % KSTEP == 0 && KSTEPS_LAST >= 1 && KSTEPS_LAST <= 4, "K steps");
};

// a work item of the uniform-tree kernel: level index, target octant, child octant (L2L),
// tile origin in slab coordinates, output half
struct WorkItem {
    int li, oct, c, px0, py0, pz0, half;
};

// the terms of a work item, in a fixed order.  M2L: the displacements v_d in
// [-3 + o_d, 2 + o_d] that are not all |v_d| <= 1 (189 of 216); M2M: the 8 child octants;
// L2L: one term.
struct Terms {
    int mode, o[3], v[3], j;
    __device__ void first(int mode_, int oct) {
        mode = mode_;
        j = 0;
        o[0] = oct & 1; o[1] = (oct >> 1) & 1; o[2] = (oct >> 2) & 1;
        v[0] = -3 + o[0]; v[1] = -3 + o[1]; v[2] = -3 + o[2];
    }
    __device__ bool next() {  // advance to the next raw term; false at the end
        if (mode == kTcM2M) return ++j < 8;
        if (mode == kTcL2L) return false;
        if (++v[2] <= 2 + o[2]) return true;
        v[2] = -3 + o[2];
        if (++v[1] <= 2 + o[1]) return true;
        v[1] = -3 + o[1];
        if (++v[0] <= 2 + o[0]) return true;
        return false;
    }
    __device__ bool valid() const {
        return mode != kTcM2L || abs(v[0]) > 1 || abs(v[1]) > 1 || abs(v[2]) > 1;
    }
    // A box start (slab coordinates and slab) and the T matrix index of the current term
    __device__ void source(const WorkItem& it, int& x, int& y, int& z, int& slab, int& key) const {
        if (mode == kTcM2L) {
            int sc[3], a[3];
            for (int d = 0; d < 3; ++d) {
                const int dd = o[d] - v[d];  // in [-2, 3]
                sc[d] = dd & 1;
                a[d] = (dd - sc[d]) >> 1;    // in {-1, 0, 1}
            }
            x = it.px0 + a[0]; y = it.py0 + a[1]; z = it.pz0 + a[2];
            slab = sc[0] | (sc[1] << 1) | (sc[2] << 2);
            key = (v[0] + 3) * 49 + (v[1] + 3) * 7 + (v[2] + 3);
        } else if (mode == kTcM2M) {
            x = it.px0; y = it.py0; z = it.pz0;
            slab = j;
            key = j;
        } else {
            x = it.px0; y = it.py0; z = it.pz0;
            slab = it.oct;
            key = it.c;
        }
    }
};


// round to the nearest TF32 value (10 explicit mantissa bits) and clear the 13 low bits, so
// that hi + lo reproduces the operand exactly as the tensor core reads it
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r & 0xFFFFE000u);
}


// ---- epilogue: one accumulator row (one box) out to global memory -----------------------------
// Columns b = b_base + j (j < NP) go out in groups of 4 with 16-byte accesses: NCP is a multiple
// of 8 and every row starts on a multiple of NCP elements, so each group starts 16-byte aligned
// in the FP32 split rows and 32-byte aligned in the FP64 row.  Value of column b < NC:
// S[j] * sc (times inv_r[b] for scaled F16 operands), plus the old value when add; columns
// NC..NCP-1 are written as zeros (they lie inside the last MMA step of a later stage, where a
// stale NaN times a zero column would still be NaN).  With add the old values of a group are
// loaded DEPTH groups ahead of its store: a load placed after a store to the same row cannot be
// moved above it by the compiler, so without the ring every column would wait one memory round
// trip.  hrow / lrow (optional) receive the TF32 split of the written values.
template <int NP, int NC, int NCP, bool H>
__device__ __forceinline__ void store_row(const float (&S)[NP], int b_base, double sc, const float* inv_r, bool add,
                                          double* orow, float* hrow, float* lrow) {
    constexpr int GW = 4, NG = NP / GW, DEPTH = 4;
    static_assert(NP % 16 == 0 && NCP % 8 == 0, "column groups");
    double2 ring[DEPTH][2];
#pragma unroll
    for (int g = 0; g < DEPTH; ++g) {
        ring[g][0] = ring[g][1] = make_double2(0.0, 0.0);
        if (add && b_base + GW * g < NCP) {
            ring[g][0] = reinterpret_cast<const double2*>(orow + b_base + GW * g)[0];
            ring[g][1] = reinterpret_cast<const double2*>(orow + b_base + GW * g)[1];
        }
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int b0 = b_base + GW * g;
        const double old[4] = {ring[g % DEPTH][0].x, ring[g % DEPTH][0].y, ring[g % DEPTH][1].x, ring[g % DEPTH][1].y};
        if (add && g + DEPTH < NG && b0 + GW * DEPTH < NCP) {
            ring[g % DEPTH][0] = reinterpret_cast<const double2*>(orow + b0 + GW * DEPTH)[0];
            ring[g % DEPTH][1] = reinterpret_cast<const double2*>(orow + b0 + GW * DEPTH)[1];
        }
        if (b0 < NCP) {
            double v[GW];
#pragma unroll
            for (int j = 0; j < GW; ++j) {
                double x = 0.0;
                if (b0 + j < NC) {
                    x = (double)S[GW * g + j] * sc;
                    if constexpr (H) x *= (double)inv_r[b0 + j];
                    if (add) x += old[j];
                }
                v[j] = x;
            }
            reinterpret_cast<double2*>(orow + b0)[0] = make_double2(v[0], v[1]);
            reinterpret_cast<double2*>(orow + b0)[1] = make_double2(v[2], v[3]);
            if (hrow) {
                float h[GW], l[GW];
#pragma unroll
                for (int j = 0; j < GW; ++j) {
                    const float f = (float)v[j];
                    h[j] = to_tf32(f);
                    l[j] = to_tf32(f - h[j]);
                }
                *reinterpret_cast<float4*>(hrow + b0) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4*>(lrow + b0) = make_float4(l[0], l[1], l[2], l[3]);
            }
        }
    }
}

}  // namespace tc

// ---- host side: tensor maps --------------------------------------------------------------------
inline PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}


// 3-D map (coef, row, matrix) over [nkey][npt][rowlen] elements (FP32, or F16 when f16) with
// boxes of 128 bytes x np rows
inline bool encode_rows(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const void* base, int rowlen, int npt,
                        int nkey, int np, bool f16 = false) {
    const cuuint64_t es_bytes = f16 ? 2 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)rowlen, (cuuint64_t)npt, (cuuint64_t)nkey};
    const cuuint64_t strides[2] = {(cuuint64_t)rowlen * es_bytes, (cuuint64_t)rowlen * es_bytes * npt};
    const cuuint32_t box[3] = {(cuuint32_t)(128 / es_bytes), (cuuint32_t)np, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base),
               dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


}  // namespace dafmm
