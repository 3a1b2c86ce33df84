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

// A wait polls try_wait (which itself suspends the thread for a while when the phase is not
// complete) with no sleep between polls: a sleep adds its own latency to every hand-off of the
// pipeline.  It is declared stuck after 1 s of device time (checked every 256 polls) or after
// kWaitPolls polls, whichever comes first.
constexpr long long kWaitPolls = 1ll << 26;
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait; on expiry records `code` in *err and returns false
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1; i < kWaitPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 0 && global_ns() - t0 > kWaitNs) break;
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

// 32 lanes x 32 columns, load and wait in one statement (half the round trips of two x16 loads)
__device__ __forceinline__ void tmem_ld32w(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {"
        "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// one term's accumulator (NP columns from tb) folded into the row sums S: S += acc (TF32), or
// S += acc * f (F16: f undoes the term's scales).  WIDE: 32 columns per load and wait instead of
// 16 -- half the round trips, 16 more registers (taken where the accumulator is narrow, in the
// harmonic basis)
template <int NP, bool H, bool WIDE>
__device__ __forceinline__ void fold_term(uint32_t tb, float f, float (&S)[NP]) {
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += (WIDE ? 32 : 16)) {
        if (WIDE && c0 + 32 <= NP) {
            uint32_t r[32];
            tmem_ld32w(tb + c0, r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if constexpr (H) S[c0 + j] = fmaf(__uint_as_float(r[j]), f, S[c0 + j]);
                else S[c0 + j] += __uint_as_float(r[j]);
            }
        } else {
#pragma unroll
            for (int c1 = c0; c1 < c0 + (WIDE ? 32 : 16) && c1 < NP; c1 += 16) {
                uint32_t r[16];
                tmem_ld16w(tb + c1, r);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if constexpr (H) S[c1 + j] = fmaf(__uint_as_float(r[j]), f, S[c1 + j]);
                    else S[c1 + j] += __uint_as_float(r[j]);
                }
            }
        }
    }
}

// 32 lanes x 16 columns from registers into TMEM (the caller waits with tmem_wait_st)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- configuration per order ------------------------------------------------------------------
// H = false: TF32 operands (rows of ncp FP32 values); H = true: F16 operands (rows of ncph =
// ncoef rounded up to 16 halves).  Either way a K chunk is 128 bytes of a row (32 TF32 or 64
// F16 values) and one MMA step takes 32 bytes of it (K = 8 or 16).  R = true: the contraction
// in the harmonic basis (the (p + 1)^2 free coefficients of rows and columns; see nharm_of).
template <int P, bool H = false, bool R = false>
struct Cfg {
    static constexpr int NC = R ? nharm_of(P) : ncoef_of(P);  // coefficients contracted and produced
    static constexpr int NCP = (NC + 7) / 8 * 8;                 // output row stride
    static constexpr int ROWLEN = H ? (NC + 15) / 16 * 16 : NCP;  // operand row length, elements
    static constexpr int KPC = H ? 64 : 32;                         // elements per 128-byte chunk
    static constexpr int KSTEP = H ? 16 : 8;                        // elements per MMA step
    static constexpr int NPF = (NC + 15) / 16 * 16;               // N padded to the MMA granule
    static constexpr int NHALF = NPF > 192 ? 2 : 1;                // N split: <= 192 register sums per thread
    static constexpr int NP = NHALF == 1 ? NPF : (NPF / 2 + 15) / 16 * 16;
    static constexpr int NPT = NHALF == 1 ? NPF : 2 * NP;         // rows per matrix in the B tables
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
    __device__ bool next_valid() {  // advance to the next valid term; false at the end
        while (next())
            if (valid()) return true;
        return false;
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
// The finished row of each of the warp's 32 lanes sits in TMEM columns tb .. tb + NP - 1; it
// goes out 16 columns per step of a loop that is not unrolled, so the code stays small: this
// runs once per tile, and a fully unrolled store of NP columns was measured to stall on
// instruction fetch for tens of microseconds.  Column b = b_base + j < NC receives S_j * sc
// (times inv_r[b] for scaled F16 operands), plus the old value when add; columns NC..NCP-1 are
// written as zeros (they lie inside the last MMA step of a later stage, where a stale NaN times
// a zero column would still be NaN).  With f32 the row holds FP32 values and the arithmetic is
// FP32 (scf = sc rounded to FP32); otherwise both are FP64, which this part executes at a small
// fraction of the FP32 rate.  Accesses are 16 bytes (NCP is a multiple of 8 and rows start on
// multiples of NCP elements); the old values (add) of the step after next and the column
// factors (F16) of the next step are requested before this step's stores.  inv_r holds at least NCP values.  hrow / lrow
// (optional) receive the TF32 split of the written values.
// All lanes call this (the TMEM loads are warp-wide); `valid` selects the lanes that own a row.
template <int NP, int NC, int NCP, bool H>
__device__ __forceinline__ void store_row(uint32_t tb, bool valid, int b_base, double sc, float scf, const float* inv_r,
                                          bool add, bool f32, void* orow, float* hrow, float* lrow) {
    static_assert(NP % 16 == 0 && NCP % 8 == 0, "column groups");
    double* od = static_cast<double*>(orow);
    float* of = static_cast<float*>(orow);
    // old values of the 16 columns from b: FP32 in o[0..3], FP64 in o[0..7]; groups at or past
    // NCP are not read
    auto load_old = [&](int b, uint4 (&o)[8]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (b + 4 * k >= NCP) continue;
            if (f32) {
                o[k] = *reinterpret_cast<const uint4*>(of + b + 4 * k);
            } else {
                o[2 * k] = reinterpret_cast<const uint4*>(od + b + 4 * k)[0];
                o[2 * k + 1] = reinterpret_cast<const uint4*>(od + b + 4 * k)[1];
            }
        }
    };
    // per-column factors of the 16 columns from b (F16 operands)
    auto load_inv = [&](int b, float4 (&f)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (b + 4 * k < NCP) f[k] = *reinterpret_cast<const float4*>(inv_r + b + 4 * k);
    };
    uint4 nxt[8], nx2[8];  // old values one and two steps ahead
    float4 nxf[4];
#pragma unroll
    for (int k = 0; k < 8; ++k) nxt[k] = nx2[k] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) nxf[k] = make_float4(1.f, 1.f, 1.f, 1.f);
    const bool rd = valid && add;
    if (rd) load_old(b_base, nxt);
    if (rd && 16 < NP && b_base + 16 < NCP) load_old(b_base + 16, nx2);
    if (H && valid && b_base < NCP) load_inv(b_base, nxf);
#pragma unroll 1
    for (int c0 = 0; c0 < NP; c0 += 16) {
        __syncwarp();
        uint32_t r[16];
        tmem_ld16w(tb + c0, r);
        const int b0 = b_base + c0;
        uint4 cur[8];
        float4 cf[4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cur[k] = nxt[k];
            nxt[k] = nx2[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cf[k] = nxf[k];
        // later steps' loads go out before this step's stores
        if (rd && c0 + 32 < NP && b0 + 32 < NCP) load_old(b0 + 32, nx2);
        if (H && valid && c0 + 16 < NP && b0 + 16 < NCP) load_inv(b0 + 16, nxf);
        if (!valid) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int bg = b0 + 4 * k;
            if (bg >= NCP) continue;
            float h[4], l[4];
            if (f32) {
                const float o4[4] = {__uint_as_float(cur[k].x), __uint_as_float(cur[k].y), __uint_as_float(cur[k].z),
                                     __uint_as_float(cur[k].w)};
                float v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float x = 0.f;
                    if (bg + j < NC) {
                        x = __uint_as_float(r[4 * k + j]) * scf;
                        if constexpr (H) x *= (&cf[k].x)[j];
                        if (add) x += o4[j];
                    }
                    v[j] = x;
                    h[j] = to_tf32(x);
                    l[j] = to_tf32(x - h[j]);
                }
                *reinterpret_cast<float4*>(of + bg) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                const double o4[4] = {__hiloint2double((int)cur[2 * k].y, (int)cur[2 * k].x),
                                      __hiloint2double((int)cur[2 * k].w, (int)cur[2 * k].z),
                                      __hiloint2double((int)cur[2 * k + 1].y, (int)cur[2 * k + 1].x),
                                      __hiloint2double((int)cur[2 * k + 1].w, (int)cur[2 * k + 1].z)};
                double v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    double x = 0.0;
                    if (bg + j < NC) {
                        x = (double)__uint_as_float(r[4 * k + j]) * sc;
                        if constexpr (H) x *= (double)(&cf[k].x)[j];
                        if (add) x += o4[j];
                    }
                    v[j] = x;
                    const float f = (float)x;
                    h[j] = to_tf32(f);
                    l[j] = to_tf32(f - h[j]);
                }
                reinterpret_cast<double2*>(od + bg)[0] = make_double2(v[0], v[1]);
                reinterpret_cast<double2*>(od + bg)[1] = make_double2(v[2], v[3]);
            }
            if (hrow) {
                *reinterpret_cast<float4*>(hrow + bg) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4*>(lrow + bg) = make_float4(l[0], l[1], l[2], l[3]);
            }
        }
    }
    __syncwarp();
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
