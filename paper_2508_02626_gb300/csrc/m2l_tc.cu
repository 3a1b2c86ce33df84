// m2l_tc.cu -- M2L (Eq. 5) on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For a target box t of level l and each of the 189 displacements v of its octant
// (Sec. 3.4), L~_t += (1/h) K^_v M~_{t-v}.  With the octant-major box layout the sources of
// 128 targets of one octant for one v form a 3-D block of one octant slab, so:
//   A (128 x K, K-major)  = that block of multipoles, gathered by one 5-D TMA box load
//                           (zero-filled where the block leaves the domain);
//   B (N x K, K-major)    = K^_v, one 3-D TMA box load;
//   D (128 x N, FP32)     = accumulated over all v in tensor memory (TMEM).
// Precision: each FP32 operand is split into TF32 high and low parts (x = hi + lo, both
// rounded to TF32), and D += A_hi B_hi + A_hi B_lo + A_lo B_hi, which carries about 22
// mantissa bits per product, with FP32 accumulation.
//
// One persistent CTA per SM walks a list of (level, octant, tile, N-half) work items.
// Warp roles: warp 0 issues TMA loads into a ring of shared-memory stages, warp 1 issues
// the MMAs (one elected thread) and owns the TMEM allocation, warps 2-5 drain the
// double-buffered accumulator (tcgen05.ld) and write L~ in FP64.  Every mbarrier wait is
// bounded: on expiry the kernel records an error flag, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "m2l_tc.h"

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

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns of TMEM into 16 registers per thread (no wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- the kernel -----------------------------------------------------------------------------
template <int P>
struct Cfg {
    static constexpr int NC = ncoef_of(P);
    static constexpr int NCP = ncp_of(P);
    static constexpr int NPF = (NC + 15) / 16 * 16;               // N padded to the MMA granule
    static constexpr int NHALF = NPF > 192 ? 2 : 1;                // N split: <= 192 register sums per thread
    static constexpr int NP = NHALF == 1 ? NPF : (NPF / 2 + 15) / 16 * 16;
    static constexpr int NKC = (NCP + 31) / 32;                    // K chunks of 32 (128 bytes)
    static constexpr int KSTEPS_LAST = (NCP - 32 * (NKC - 1)) / 8; // K steps of 8 in the last chunk
    static constexpr int A_BYTES = 128 * 128;
    static constexpr int B_BYTES = NP * 128;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int SMEM_AVAIL = 227 * 1024 - 2048;
    static constexpr int STAGES = (SMEM_AVAIL / STAGE_BYTES) > 4 ? 4 : (SMEM_AVAIL / STAGE_BYTES);
    static constexpr int TMEM_COLS = 2 * NP <= 256 ? 256 : 512;
    static constexpr uint32_t IDESC = idesc_tf32(128, NP);
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= 192, "MMA N");
    static_assert(STAGES >= 2, "pipeline depth");
    static_assert(2 * NP <= TMEM_COLS, "TMEM double buffer");
};

struct WorkItem {
    int li, oct, px0, py0, pz0, half;
};

__device__ __forceinline__ WorkItem decode(const M2LTCParams& prm, int w) {
    WorkItem it;
    int li = 0;
    while (li + 1 < prm.nlev && w >= prm.tile_base[li + 1]) ++li;
    int local = w - prm.tile_base[li];
    it.li = li;
    it.half = local % prm.nhalf;
    local /= prm.nhalf;
    it.oct = local & 7;
    local >>= 3;
    const int P = prm.P[li], bx = prm.bx[li], by = prm.by[li];
    const int nx = P / bx, ny = P / by;
    it.px0 = (local % nx) * bx;
    it.py0 = ((local / nx) % ny) * by;
    it.pz0 = (local / (nx * ny)) * prm.bz[li];
    return it;
}

// the 189 displacements of a target octant, in a fixed order: v_d in [-3 + o_d, 2 + o_d], not all |v_d| <= 1
struct VIter {
    int o[3];
    int v[3];
    __device__ void first(int oct) {
        o[0] = oct & 1; o[1] = (oct >> 1) & 1; o[2] = (oct >> 2) & 1;
        v[0] = -3 + o[0]; v[1] = -3 + o[1]; v[2] = -3 + o[2];
    }
    __device__ bool next() {  // advance to the next raw combination; false at the end
        if (++v[2] <= 2 + o[2]) return true;
        v[2] = -3 + o[2];
        if (++v[1] <= 2 + o[1]) return true;
        v[1] = -3 + o[1];
        if (++v[0] <= 2 + o[0]) return true;
        return false;
    }
    __device__ bool valid() const { return abs(v[0]) > 1 || abs(v[1]) > 1 || abs(v[2]) > 1; }
};

template <int P>
__global__ void __launch_bounds__(192, 1) k_m2l_tc(const __grid_constant__ M2LTCParams prm) {
    using C = Cfg<P>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage ring, then barriers
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* bar_area = base + C::STAGES * C::STAGE_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(bar_area);
    uint64_t* empty = full + C::STAGES;
    uint64_t* acc_full = empty + C::STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), 128);
        }
        mbar_init(smem_u32(drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        for (int l = 0; l < prm.nlev; ++l) {
            prefetch_map(&prm.a_hi[l]);
            prefetch_map(&prm.a_lo[l]);
        }
        prefetch_map(&prm.b_hi);
        prefetch_map(&prm.b_lo);
        int stage = 0;
        uint32_t phase = 0;
        int armed[C::STAGES];  // parity of the last phase armed on each full barrier, -1 if none
        for (int s = 0; s < C::STAGES; ++s) armed[s] = -1;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const WorkItem it = decode(prm, w);
            const uint32_t a_bytes = 128u * prm.bx[it.li] * prm.by[it.li] * prm.bz[it.li];
            VIter vi;
            vi.first(it.oct);
            do {
                if (!vi.valid()) continue;
                int sc[3], a[3];
                for (int d = 0; d < 3; ++d) {
                    const int dd = vi.o[d] - vi.v[d];  // in [-2, 3]
                    sc[d] = dd & 1;
                    a[d] = (dd - sc[d]) >> 1;          // in {-1, 0, 1}
                }
                const int soct = sc[0] | (sc[1] << 1) | (sc[2] << 2);
                const int key = (vi.v[0] + 3) * 49 + (vi.v[1] + 3) * 7 + (vi.v[2] + 3);
                for (int kc = 0; kc < C::NKC && ok; ++kc) {
                    ok = mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, prm.err, 11);
                    if (!ok) break;
                    unsigned char* st = base + stage * C::STAGE_BYTES;
                    const uint32_t fb = smem_u32(&full[stage]);
                    mbar_expect_tx(fb, 2u * a_bytes + 2u * C::B_BYTES);
                    armed[stage] = (int)phase;
                    tma_load_5d(smem_u32(st), &prm.a_hi[it.li], fb, kc * 32, it.px0 + a[0], it.py0 + a[1], it.pz0 + a[2], soct);
                    tma_load_5d(smem_u32(st + C::A_BYTES), &prm.a_lo[it.li], fb, kc * 32, it.px0 + a[0], it.py0 + a[1],
                                it.pz0 + a[2], soct);
                    tma_load_3d(smem_u32(st + 2 * C::A_BYTES), &prm.b_hi, fb, kc * 32, it.half * C::NP, key);
                    tma_load_3d(smem_u32(st + 2 * C::A_BYTES + C::B_BYTES), &prm.b_lo, fb, kc * 32, it.half * C::NP, key);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            } while (vi.next() && ok);
        }
        // wait (bounded) until every copy this thread armed has landed before the block may exit
        for (int s = 0; s < C::STAGES; ++s)
            if (armed[s] >= 0) mbar_wait(smem_u32(&full[s]), (uint32_t)armed[s], prm.err, 12);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        // one fresh accumulator per displacement v (alternating TMEM buffers): at most
        // 3 * ceil(ncoef/8) MMA accumulation steps land in one FP32 accumulator
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acc_ph[2] = {0, 0};
        bool ok = true;
        int uses = 0;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const WorkItem it = decode(prm, w);
            VIter vi;
            vi.first(it.oct);
            do {
                if (!vi.valid()) continue;
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_empty[buf]), acc_ph[buf] ^ 1u, prm.err, 21);
                if (!ok) break;
                acc_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t d = tmem_base + (uint32_t)(buf * C::NP);
                uint32_t accum = 0;
                for (int kc = 0; kc < C::NKC && ok; ++kc) {
                    ok = mbar_wait(smem_u32(&full[stage]), phase, prm.err, 22);
                    if (!ok) break;
                    fence_after_sync();
                    const uint32_t st = smem_u32(base + stage * C::STAGE_BYTES);
                    const int nks = (kc == C::NKC - 1) ? C::KSTEPS_LAST : 4;
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t ah = smem_desc_sw128(st + ks * 32);
                        const uint64_t al = smem_desc_sw128(st + C::A_BYTES + ks * 32);
                        const uint64_t bh = smem_desc_sw128(st + 2 * C::A_BYTES + ks * 32);
                        const uint64_t bl = smem_desc_sw128(st + 2 * C::A_BYTES + C::B_BYTES + ks * 32);
                        mma_tf32(d, ah, bl, C::IDESC, accum);  // small cross terms first
                        accum = 1;
                        mma_tf32(d, al, bh, C::IDESC, 1);
                        mma_tf32(d, ah, bh, C::IDESC, 1);
                    }
                    mma_commit(smem_u32(&empty[stage]));
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (ok) mma_commit(smem_u32(&acc_full[buf]));
                ++uses;
            } while (vi.next() && ok);
        }
        // every MMA this thread issued has finished once the drain barrier flips
        mma_commit(smem_u32(drain));
        mbar_wait(smem_u32(drain), 0, prm.err, 23);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        // sums the per-displacement accumulators of its row in FP32 registers (CUDA cores)
        const int q = warp & 3;          // TMEM lane quarter of this warp
        const int row = 32 * q + lane;   // accumulator row = target within the tile
        uint32_t accf_ph[2] = {0, 0};
        int uses = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const WorkItem it = decode(prm, w);
            float S[C::NP];
#pragma unroll
            for (int j = 0; j < C::NP; ++j) S[j] = 0.f;
            VIter vi;
            vi.first(it.oct);
            do {
                if (!vi.valid()) continue;
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_full[buf]), accf_ph[buf], prm.err, 31);
                if (!ok) break;
                accf_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t tb = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::NP);
#pragma unroll
                for (int c0 = 0; c0 < C::NP; c0 += 32) {
                    uint32_t r0[16], r1[16];
                    tmem_ld16(tb + c0, r0);
                    if (c0 + 16 < C::NP) tmem_ld16(tb + c0 + 16, r1);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) S[c0 + j] += __uint_as_float(r0[j]);
                    if (c0 + 16 < C::NP) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) S[c0 + 16 + j] += __uint_as_float(r1[j]);
                    }
                }
                fence_before_sync();
                mbar_arrive(smem_u32(&acc_empty[buf]));
                ++uses;
            } while (vi.next() && ok);
            if (!ok) break;
            const int bx = prm.bx[it.li], by = prm.by[it.li], bz = prm.bz[it.li];
            if (row < bx * by * bz) {
                const int Pl = prm.P[it.li];
                const int x = row % bx, y = (row / bx) % by, z = row / (bx * by);
                const int t = it.oct * Pl * Pl * Pl + ((it.pz0 + z) * Pl + (it.py0 + y)) * Pl + (it.px0 + x);
                double* Lrow = prm.L[it.li] + (size_t)t * C::NCP;
                const double ih = prm.inv_h[it.li];
#pragma unroll
                for (int j = 0; j < C::NP; ++j) {
                    const int b = it.half * C::NP + j;
                    if (b < C::NC) Lrow[b] = (double)S[j] * ih;
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::TMEM_COLS)
                     : "memory");
    }
}

// ---- split of FP64 data into TF32 high/low parts ----------------------------------------------
// round to the nearest TF32 value (10 explicit mantissa bits) and clear the 13 low bits, so
// that hi + lo reproduces the operand exactly as the tensor core reads it
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r & 0xFFFFE000u);
}

__global__ void k_split_tf32(const double* __restrict__ src, float* __restrict__ hi, float* __restrict__ lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = src[i];
        const float h = to_tf32((float)x);
        hi[i] = h;
        lo[i] = to_tf32((float)(x - (double)h));
    }
}

// K^ split, rows padded from nc to npt (zero rows), [343][npt][ncp]
__global__ void k_split_k(const double* __restrict__ K64, int nc, int ncp, int npt, float* __restrict__ hi,
                          float* __restrict__ lo) {
    const size_t n = (size_t)kNumKeys * npt * ncp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(i % ncp);
        const size_t rk = i / ncp;
        const int b = (int)(rk % npt);
        const size_t key = rk / npt;
        double x = 0.0;
        if (b < nc) x = K64[(key * nc + b) * ncp + a];
        const float h = to_tf32((float)x);
        hi[i] = h;
        lo[i] = to_tf32((float)(x - (double)h));
    }
}

}  // namespace tc

// ---- host side ---------------------------------------------------------------------------------
int m2l_tc_npt(int p) {
    const int nc = ncoef_of(p);
    const int npf = (nc + 15) / 16 * 16;
    if (npf <= 192) return npf;
    return 2 * ((npf / 2 + 15) / 16 * 16);
}

cudaError_t m2l_tc_split_tf32(const double* src, float* hi, float* lo, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    tc::k_split_tf32<<<blocks, 256, 0, s>>>(src, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t m2l_tc_split_k(const double* K64, int p, float* hi, float* lo, cudaStream_t s) {
    const int nc = ncoef_of(p), ncp = ncp_of(p), npt = m2l_tc_npt(p);
    tc::k_split_k<<<152 * 16, 256, 0, s>>>(K64, nc, ncp, npt, hi, lo);
    return cudaGetLastError();
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

template <int P>
static cudaError_t launch_tc(const M2LTCArgs& a, cudaStream_t s) {
    using C = tc::Cfg<P>;
    auto encode = get_encode();
    if (!encode) return cudaErrorNotSupported;
    M2LTCParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.nlev = 0;
    prm.nhalf = C::NHALF;
    prm.err = a.err;
    int tiles = 0;
    // finest level first: all work items cost the same, the list is only an order
    for (int l = a.lmax; l >= a.lmin; --l) {
        const int li = prm.nlev++;
        const int Pp = 1 << (l - 1);
        int bx = Pp < 128 ? Pp : 128;
        int by = Pp < 128 / bx ? Pp : 128 / bx;
        int bz = Pp < 128 / (bx * by) ? Pp : 128 / (bx * by);
        if (bz < 1) bz = 1;
        prm.P[li] = Pp; prm.bx[li] = bx; prm.by[li] = by; prm.bz[li] = bz;
        prm.L[li] = a.L[l];
        prm.inv_h[li] = a.inv_h[l];
        const int tpo = (Pp / bx) * (Pp / by) * (Pp / bz);
        prm.tile_base[li] = tiles;
        tiles += 8 * tpo * C::NHALF;
        const cuuint64_t dims[5] = {(cuuint64_t)C::NCP, (cuuint64_t)Pp, (cuuint64_t)Pp, (cuuint64_t)Pp, 8};
        const cuuint64_t row = (cuuint64_t)C::NCP * 4;
        const cuuint64_t strides[4] = {row, row * Pp, row * Pp * Pp, row * Pp * Pp * Pp};
        const cuuint32_t box[5] = {32, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        for (int h = 0; h < 2; ++h) {
            CUresult r = encode(h == 0 ? &prm.a_hi[li] : &prm.a_lo[li], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5,
                                (void*)(h == 0 ? a.Mhi[l] : a.Mlo[l]), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    prm.tile_base[prm.nlev] = tiles;
    prm.ntiles = tiles;
    {
        const int npt = m2l_tc_npt(P);
        const cuuint64_t dims[3] = {(cuuint64_t)C::NCP, (cuuint64_t)npt, (cuuint64_t)kNumKeys};
        const cuuint64_t strides[2] = {(cuuint64_t)C::NCP * 4, (cuuint64_t)C::NCP * 4 * npt};
        const cuuint32_t box[3] = {32, (cuuint32_t)C::NP, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        for (int h = 0; h < 2; ++h) {
            CUresult r = encode(h == 0 ? &prm.b_hi : &prm.b_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                (void*)(h == 0 ? a.Khi : a.Klo), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc::k_m2l_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tiles < a.num_sms ? tiles : a.num_sms;
    tc::k_m2l_tc<P><<<grid, 192, C::SMEM_BYTES, s>>>(prm);
    return cudaGetLastError();
}

cudaError_t m2l_tc_launch(int p, const M2LTCArgs& a, cudaStream_t s) {
    switch (p) {
        case 2: return launch_tc<2>(a, s);
        case 3: return launch_tc<3>(a, s);
        case 4: return launch_tc<4>(a, s);
        case 5: return launch_tc<5>(a, s);
        case 6: return launch_tc<6>(a, s);
        case 7: return launch_tc<7>(a, s);
        case 8: return launch_tc<8>(a, s);
        case 9: return launch_tc<9>(a, s);
        case 10: return launch_tc<10>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dafmm
