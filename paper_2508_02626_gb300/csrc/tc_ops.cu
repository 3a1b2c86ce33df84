// tc_ops.cu -- the dense contractions of the FMM on the 5th-generation tensor cores
// (tcgen05, sm_103a): M2L (Eq. 5), M2M (Eq. 4) and L2L (Eq. 7).
//
// All three are sums of small dense products  out_t (+)= scale * sum_j T_j A_{s(t,j)}  over
// boxes t, with box-scaled expansions and level-independent matrices T_j:
//   M2L  T_j = K^_v for the 189 displacements v of the target's octant (Sec. 3.4),
//        A = multipoles of the sources t - v, out = locals of level l (written), scale 1/h;
//   M2M  T_j = M2M table of child octant j (8 terms, Sec. 3.3 octant maps),
//        A = multipoles of the children, out = parent multipoles (written);
//   L2L  T = L2L table of the child octant (1 term), A = parent locals,
//        out = child locals (added to what M2L wrote).
// With the octant-major box layout the A rows of 128 boxes of one tile form a 3-D block of
// one octant slab: one 5-D TMA box load (zero-filled outside the domain).  T is one 3-D
// box.  Each FP32 operand is split into TF32 parts x = hi + lo and the product takes
// A_hi T_lo + A_lo T_hi + A_hi T_hi (about 22 mantissa bits per product) into a fresh
// FP32 TMEM accumulator per term (double-buffered); the epilogue warps add the terms in
// FP32 registers, write the FP64 result and, when asked, its TF32 split for the next
// stage.
//
// One persistent CTA per SM walks the work items.  Warp roles: warp 0 issues TMA loads
// into a ring of shared-memory stages, warp 1 issues the MMAs (one elected thread) and
// owns the TMEM allocation, warps 2-5 drain the accumulators.  Every mbarrier wait is
// bounded: on expiry the kernel records an error flag, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc_ops.h"
#include "tree_common.cuh"

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

// ---- work items and their terms ---------------------------------------------------------------
struct WorkItem {
    int li, oct, c, px0, py0, pz0, half;
};

__device__ __forceinline__ WorkItem decode(const TCParams& prm, int w) {
    WorkItem it;
    int li = 0;
    while (li + 1 < prm.nlev && w >= prm.tile_base[li + 1]) ++li;
    int local = w - prm.tile_base[li];
    it.li = li;
    it.half = local % prm.nhalf;
    local /= prm.nhalf;
    it.oct = 0;
    it.c = 0;
    if (prm.mode == kTcM2L || prm.mode == kTcL2L) {
        it.oct = local & 7;
        local >>= 3;
    }
    if (prm.mode == kTcL2L) {
        it.c = local & 7;
        local >>= 3;
    }
    const int S = prm.S[li], bx = prm.bx[li], by = prm.by[li];
    const int nx = S / bx, ny = S / by;
    it.px0 = (local % nx) * bx;
    it.py0 = ((local / nx) % ny) * by;
    it.pz0 = (local / (nx * ny)) * prm.bz[li];
    return it;
}

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

// output box index of tile row (x, y, z) of a work item
__device__ __forceinline__ int out_index(const TCParams& prm, const WorkItem& it, int x, int y, int z) {
    const int S = prm.S[it.li];
    const int px = it.px0 + x, py = it.py0 + y, pz = it.pz0 + z;
    if (prm.mode == kTcM2L) return it.oct * S * S * S + (pz * S + py) * S + px;
    if (prm.mode == kTcM2M) return octmajor_index(prm.out_level[it.li], px, py, pz);
    // L2L: parent (2q + o) at the parent level, child 2 (2q + o) + c at the output level
    const int ox = it.oct & 1, oy = (it.oct >> 1) & 1, oz = (it.oct >> 2) & 1;
    const int Pl = 1 << (prm.out_level[it.li] - 1);
    const int cx = 2 * px + ox, cy = 2 * py + oy, cz = 2 * pz + oz;
    return it.c * Pl * Pl * Pl + (cz * Pl + cy) * Pl + cx;
}

__device__ __forceinline__ float to_tf32(float x);

// ---- the kernel -----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(192, 1) k_tc(const __grid_constant__ TCParams prm) {
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
            Terms tm;
            tm.first(prm.mode, it.oct);
            do {
                if (!tm.valid()) continue;
                int sx, sy, sz, slab, key;
                tm.source(it, sx, sy, sz, slab, key);
                for (int kc = 0; kc < C::NKC && ok; ++kc) {
                    ok = mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, prm.err, 11);
                    if (!ok) break;
                    unsigned char* st = base + stage * C::STAGE_BYTES;
                    const uint32_t fb = smem_u32(&full[stage]);
                    mbar_expect_tx(fb, 2u * a_bytes + 2u * C::B_BYTES);
                    armed[stage] = (int)phase;
                    tma_load_5d(smem_u32(st), &prm.a_hi[it.li], fb, kc * 32, sx, sy, sz, slab);
                    tma_load_5d(smem_u32(st + C::A_BYTES), &prm.a_lo[it.li], fb, kc * 32, sx, sy, sz, slab);
                    tma_load_3d(smem_u32(st + 2 * C::A_BYTES), &prm.b_hi, fb, kc * 32, it.half * C::NP, key);
                    tma_load_3d(smem_u32(st + 2 * C::A_BYTES + C::B_BYTES), &prm.b_lo, fb, kc * 32, it.half * C::NP, key);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            } while (tm.next() && ok);
        }
        // wait (bounded) until every copy this thread armed has landed before the block may exit
        for (int s = 0; s < C::STAGES; ++s)
            if (armed[s] >= 0) mbar_wait(smem_u32(&full[s]), (uint32_t)armed[s], prm.err, 12);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        // one fresh accumulator per term (alternating TMEM buffers): at most
        // 3 * ceil(ncoef/8) MMA accumulation steps land in one FP32 accumulator
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acc_ph[2] = {0, 0};
        bool ok = true;
        int uses = 0;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const WorkItem it = decode(prm, w);
            Terms tm;
            tm.first(prm.mode, it.oct);
            do {
                if (!tm.valid()) continue;
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
            } while (tm.next() && ok);
        }
        // every MMA this thread issued has finished once the drain barrier flips
        mma_commit(smem_u32(drain));
        mbar_wait(smem_u32(drain), 0, prm.err, 23);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;          // TMEM lane quarter of this warp
        const int row = 32 * q + lane;   // accumulator row = box within the tile
        uint32_t accf_ph[2] = {0, 0};
        int uses = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const WorkItem it = decode(prm, w);
            float S[C::NP];
#pragma unroll
            for (int j = 0; j < C::NP; ++j) S[j] = 0.f;
            Terms tm;
            tm.first(prm.mode, it.oct);
            do {
                if (!tm.valid()) continue;
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_full[buf]), accf_ph[buf], prm.err, 31);
                if (!ok) break;
                accf_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t tb = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::NP);
#pragma unroll
                for (int c0 = 0; c0 < C::NP; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16w(tb + c0, r);
#pragma unroll
                    for (int j = 0; j < 16; ++j) S[c0 + j] += __uint_as_float(r[j]);
                }
                fence_before_sync();
                mbar_arrive(smem_u32(&acc_empty[buf]));
                ++uses;
            } while (tm.next() && ok);
            if (!ok) break;
            const int bx = prm.bx[it.li], by = prm.by[it.li], bz = prm.bz[it.li];
            if (row < bx * by * bz) {
                const int x = row % bx, y = (row / bx) % by, z = row / (bx * by);
                const size_t t = (size_t)out_index(prm, it, x, y, z) * C::NCP;
                double* orow = prm.out[it.li] + t;
                float* hrow = prm.out_hi[it.li] ? prm.out_hi[it.li] + t : nullptr;
                float* lrow = prm.out_lo[it.li] ? prm.out_lo[it.li] + t : nullptr;
                const double sc = prm.scale[it.li];
                const bool add = prm.mode == kTcL2L;
#pragma unroll
                for (int j = 0; j < C::NP; ++j) {
                    const int b = it.half * C::NP + j;
                    if (b < C::NC) {
                        double v = (double)S[j] * sc;
                        if (add) v += orow[b];
                        orow[b] = v;
                        if (hrow) {
                            const float f = (float)v;
                            const float h = to_tf32(f);
                            hrow[b] = h;
                            lrow[b] = to_tf32(f - h);
                        }
                    } else if (b < C::NCP) {
                        // padding columns lie inside the last MMA K step of the next stage:
                        // they must hold zeros (a stale NaN times a zero column is NaN)
                        orow[b] = 0.0;
                        if (hrow) {
                            hrow[b] = 0.f;
                            lrow[b] = 0.f;
                        }
                    }
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

// ---- gathered M2L: adaptive trees and forests ---------------------------------------------------
// Same pipeline as k_tc, but the A rows (source multipoles) of a 128-target tile are gathered
// one 16-byte chunk at a time with cp.async into the 128-byte-swizzled K-major layout that a
// TMA box would produce (chunk j of row r at (r / 8) * 1024 + (r % 8) * 128 + (j ^ r % 8) * 16),
// zero-filled for missing sources and for columns past ncp.  The whole producer warp gathers;
// its lane 0 also loads the K^_v tile by TMA.  A stage is signalled full once the TMA bytes
// have landed and every producer lane has seen its own copies complete, fenced them for the
// async proxy and arrived (33 arrivals: 32 lanes + the expect_tx arrival).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct GItem {
    int g, tile, half;
};

__device__ __forceinline__ GItem gdecode(const TCGParams& prm, int w) {
    int lo = 0, hi = prm.ngroups - 1;  // last group whose first tile is <= w
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (prm.tile_base[m] <= w) lo = m;
        else hi = m - 1;
    }
    GItem it;
    it.g = lo;
    const int local = w - prm.tile_base[lo];
    it.half = local % prm.nhalf;
    it.tile = local / prm.nhalf;
    return it;
}

// source box of target t for the displacement term `tm` (the parent's colleague at offset a,
// its child sc, with o - v = 2a + sc), or -1
__device__ __forceinline__ int m2l_source(const TCGParams& prm, int t, const Terms& tm) {
    if (t < 0) return -1;
    int sc = 0, slot = 0;
    for (int d = 0; d < 3; ++d) {
        const int dd = tm.o[d] - tm.v[d];
        const int c = dd & 1;
        const int a = (dd - c) >> 1;
        sc |= c << d;
        slot = slot * 3 + (a + 1);
    }
    const int Q = prm.colleague[27 * prm.parent[t] + slot];
    return Q >= 0 ? prm.child[8 * Q + sc] : -1;
}

template <int P>
__global__ void __launch_bounds__(192, 1) k_tcg(const __grid_constant__ TCGParams prm) {
    using C = Cfg<P>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
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
            mbar_init(smem_u32(&full[s]), 33);
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

    if (warp == 0) {
        // ---------------- gather producer (whole warp) + TMA of the matrices (lane 0) -------------
        if (lane == 0) {
            prefetch_map(&prm.b_hi);
            prefetch_map(&prm.b_lo);
        }
        int stage = 0;
        uint32_t phase = 0;
        int pend = -1;  // stage whose copies are committed but not yet signalled
        int armed[C::STAGES];
        for (int s = 0; s < C::STAGES; ++s) armed[s] = -1;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const GItem it = gdecode(prm, w);
            const int start = prm.grp_start[it.g] + it.tile * 128;
            const int cnt = min(128, prm.grp_count[it.g] - it.tile * 128);
            int tgt[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = lane + 32 * i;
                tgt[i] = r < cnt ? prm.tg[start + r] : -1;
            }
            Terms tm;
            tm.first(kTcM2L, prm.grp_oct[it.g]);
            do {
                if (!tm.valid()) continue;
                int src[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) src[i] = m2l_source(prm, tgt[i], tm);
                const int key = (tm.v[0] + 3) * 49 + (tm.v[1] + 3) * 7 + (tm.v[2] + 3);
                for (int kc = 0; kc < C::NKC; ++kc) {
                    int got = 1;
                    if (lane == 0) got = mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, prm.err, 41) ? 1 : 0;
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (!got) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = base + stage * C::STAGE_BYTES;
                    if (lane == 0) {
                        const uint32_t fb = smem_u32(&full[stage]);
                        mbar_expect_tx(fb, 2u * C::B_BYTES);
                        armed[stage] = (int)phase;
                        tma_load_3d(smem_u32(st + 2 * C::A_BYTES), &prm.b_hi, fb, kc * 32, it.half * C::NP, key);
                        tma_load_3d(smem_u32(st + 2 * C::A_BYTES + C::B_BYTES), &prm.b_lo, fb, kc * 32,
                                    it.half * C::NP, key);
                    }
                    const uint32_t sa = smem_u32(st);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = lane + 32 * i;
                        const size_t rowoff = src[i] >= 0 ? (size_t)src[i] * C::NCP : 0;
                        const uint32_t rbase = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = kc * 32 + j * 4;
                            const bool have = src[i] >= 0 && col < C::NCP;
                            const size_t e = have ? rowoff + col : 0;
                            const uint32_t off = rbase + (uint32_t)(((j ^ (r & 7)) & 7) << 4);
                            cp_async16(sa + off, prm.a_hi + e, have ? 16u : 0u);
                            cp_async16(sa + C::A_BYTES + off, prm.a_lo + e, have ? 16u : 0u);
                        }
                    }
                    cp_async_commit();
                    if (pend >= 0) {
                        cp_async_wait<1>();
                        fence_proxy_async_smem();
                        mbar_arrive(smem_u32(&full[pend]));
                    }
                    pend = stage;
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            } while (ok && tm.next());
        }
        if (pend >= 0) {
            cp_async_wait<0>();
            fence_proxy_async_smem();
            mbar_arrive(smem_u32(&full[pend]));
        }
        // every copy this warp armed must have landed before the block may exit
        if (lane == 0)
            for (int s = 0; s < C::STAGES; ++s)
                if (armed[s] >= 0) mbar_wait(smem_u32(&full[s]), (uint32_t)armed[s], prm.err, 42);
        __syncwarp();
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acc_ph[2] = {0, 0};
        bool ok = true;
        int uses = 0;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const GItem it = gdecode(prm, w);
            Terms tm;
            tm.first(kTcM2L, prm.grp_oct[it.g]);
            do {
                if (!tm.valid()) continue;
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_empty[buf]), acc_ph[buf] ^ 1u, prm.err, 43);
                if (!ok) break;
                acc_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t d = tmem_base + (uint32_t)(buf * C::NP);
                uint32_t accum = 0;
                for (int kc = 0; kc < C::NKC && ok; ++kc) {
                    ok = mbar_wait(smem_u32(&full[stage]), phase, prm.err, 44);
                    if (!ok) break;
                    fence_after_sync();
                    const uint32_t st = smem_u32(base + stage * C::STAGE_BYTES);
                    const int nks = (kc == C::NKC - 1) ? C::KSTEPS_LAST : 4;
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t ah = smem_desc_sw128(st + ks * 32);
                        const uint64_t al = smem_desc_sw128(st + C::A_BYTES + ks * 32);
                        const uint64_t bh = smem_desc_sw128(st + 2 * C::A_BYTES + ks * 32);
                        const uint64_t bl = smem_desc_sw128(st + 2 * C::A_BYTES + C::B_BYTES + ks * 32);
                        mma_tf32(d, ah, bl, C::IDESC, accum);
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
            } while (tm.next() && ok);
        }
        mma_commit(smem_u32(drain));
        mbar_wait(smem_u32(drain), 0, prm.err, 45);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;
        const int row = 32 * q + lane;
        uint32_t accf_ph[2] = {0, 0};
        int uses = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const GItem it = gdecode(prm, w);
            float S[C::NP];
#pragma unroll
            for (int j = 0; j < C::NP; ++j) S[j] = 0.f;
            Terms tm;
            tm.first(kTcM2L, prm.grp_oct[it.g]);
            do {
                if (!tm.valid()) continue;
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_full[buf]), accf_ph[buf], prm.err, 46);
                if (!ok) break;
                accf_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t tb = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::NP);
#pragma unroll
                for (int c0 = 0; c0 < C::NP; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16w(tb + c0, r);
#pragma unroll
                    for (int j = 0; j < 16; ++j) S[c0 + j] += __uint_as_float(r[j]);
                }
                fence_before_sync();
                mbar_arrive(smem_u32(&acc_empty[buf]));
                ++uses;
            } while (tm.next() && ok);
            if (!ok) break;
            const int cnt = min(128, prm.grp_count[it.g] - it.tile * 128);
            if (row < cnt) {
                const int t = prm.tg[prm.grp_start[it.g] + it.tile * 128 + row];
                double* orow = prm.out + (size_t)t * C::NCP;
                const double sc = 1.0 / prm.geom[t].w;
#pragma unroll
                for (int j = 0; j < C::NP; ++j) {
                    const int b = it.half * C::NP + j;
                    if (b < C::NC) orow[b] = (double)S[j] * sc;
                    else if (b < C::NCP) orow[b] = 0.0;
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

// a [nkey][nc][ncp] FP64 table into TF32 parts with rows padded from nc to npt (zero rows)
__global__ void k_split_rows(const double* __restrict__ K64, int nkey, int nc, int ncp, int npt, float* __restrict__ hi,
                             float* __restrict__ lo) {
    const size_t n = (size_t)nkey * npt * ncp;
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
int tc_npt(int p) {
    const int nc = ncoef_of(p);
    const int npf = (nc + 15) / 16 * 16;
    if (npf <= 192) return npf;
    return 2 * ((npf / 2 + 15) / 16 * 16);
}

cudaError_t tc_split_tf32(const double* src, float* hi, float* lo, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    tc::k_split_tf32<<<blocks, 256, 0, s>>>(src, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t tc_split_rows(const double* src, int nkey, int p, float* hi, float* lo, cudaStream_t s) {
    const int nc = ncoef_of(p), ncp = ncp_of(p), npt = tc_npt(p);
    tc::k_split_rows<<<152 * 16, 256, 0, s>>>(src, nkey, nc, ncp, npt, hi, lo);
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

// tile geometry over an S x S x S block grid: 128 boxes per tile when S^3 >= 128
static void tile_shape(int S, int& bx, int& by, int& bz) {
    bx = S < 128 ? S : 128;
    by = S < 128 / bx ? S : 128 / bx;
    bz = S < 128 / (bx * by) ? S : 128 / (bx * by);
    if (bz < 1) bz = 1;
}

// 5-D map (coef, x, y, z, slab) over an octant-major level with S slab positions per axis
static bool encode_level(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const float* base, int ncp, int S,
                         int bx, int by, int bz) {
    const cuuint64_t dims[5] = {(cuuint64_t)ncp, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)S, 8};
    const cuuint64_t row = (cuuint64_t)ncp * 4;
    const cuuint64_t strides[4] = {row, row * S, row * S * S, row * S * S * S};
    const cuuint32_t box[5] = {32, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// 3-D map (coef, row, matrix) over [nkey][npt][ncp] with boxes of np rows
static bool encode_rows(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const float* base, int ncp, int npt,
                        int nkey, int np) {
    const cuuint64_t dims[3] = {(cuuint64_t)ncp, (cuuint64_t)npt, (cuuint64_t)nkey};
    const cuuint64_t strides[2] = {(cuuint64_t)ncp * 4, (cuuint64_t)ncp * 4 * npt};
    const cuuint32_t box[3] = {32, (cuuint32_t)np, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int P>
static cudaError_t launch_tc(const TCArgs& a, cudaStream_t s) {
    using C = tc::Cfg<P>;
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    TCParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.mode = a.mode;
    prm.nhalf = C::NHALF;
    prm.err = a.err;
    int tiles = 0;
    const int per_tile_groups = a.mode == kTcM2L ? 8 : (a.mode == kTcL2L ? 64 : 1);
    // finest level first: all work items of a launch cost about the same
    for (int l = a.lmax; l >= a.lmin; --l) {
        const int li = prm.nlev++;
        // A lives on level `src` with S slab positions per axis; the tile grid is the same grid
        const int src = a.mode == kTcL2L ? l - 1 : l;
        const int S = 1 << (src - 1);
        int bx, by, bz;
        tile_shape(S, bx, by, bz);
        prm.S[li] = S; prm.bx[li] = bx; prm.by[li] = by; prm.bz[li] = bz;
        prm.out[li] = a.out[l];
        prm.out_hi[li] = a.out_hi[l];
        prm.out_lo[li] = a.out_lo[l];
        prm.scale[li] = a.scale[l];
        prm.out_level[li] = a.mode == kTcM2M ? l - 1 : l;
        prm.tile_base[li] = tiles;
        tiles += per_tile_groups * (S / bx) * (S / by) * (S / bz) * C::NHALF;
        if (!encode_level(enc, &prm.a_hi[li], a.a_hi[src], C::NCP, S, bx, by, bz) ||
            !encode_level(enc, &prm.a_lo[li], a.a_lo[src], C::NCP, S, bx, by, bz))
            return cudaErrorInvalidValue;
    }
    prm.tile_base[prm.nlev] = tiles;
    prm.ntiles = tiles;
    const int npt = tc_npt(P);
    if (!encode_rows(enc, &prm.b_hi, a.b_hi, C::NCP, npt, a.nkey, C::NP) ||
        !encode_rows(enc, &prm.b_lo, a.b_lo, C::NCP, npt, a.nkey, C::NP))
        return cudaErrorInvalidValue;
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc::k_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tiles < a.num_sms ? tiles : a.num_sms;
    tc::k_tc<P><<<grid, 192, C::SMEM_BYTES, s>>>(prm);
    return cudaGetLastError();
}

template <int P>
static cudaError_t launch_tcg(const TCGArgs& a, cudaStream_t s) {
    using C = tc::Cfg<P>;
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    if (a.ngroups > kTcgMaxGroups) return cudaErrorInvalidValue;
    TCGParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.a_hi = a.a_hi;
    prm.a_lo = a.a_lo;
    prm.tg = a.tg;
    prm.parent = a.parent;
    prm.colleague = a.colleague;
    prm.child = a.child;
    prm.geom = a.geom;
    prm.out = a.out;
    prm.nhalf = C::NHALF;
    prm.err = a.err;
    int tiles = 0, ng = 0;
    for (int g = 0; g < a.ngroups; ++g) {
        if (a.grp_count[g] <= 0) continue;  // only non-empty groups (the decode relies on it)
        prm.grp_start[ng] = a.grp_start[g];
        prm.grp_count[ng] = a.grp_count[g];
        prm.grp_oct[ng] = a.grp_oct[g];
        prm.tile_base[ng] = tiles;
        tiles += (a.grp_count[g] + 127) / 128 * C::NHALF;
        ++ng;
    }
    prm.tile_base[ng] = tiles;
    prm.ngroups = ng;
    prm.ntiles = tiles;
    if (tiles == 0) return cudaSuccess;
    const int npt = tc_npt(P);
    if (!encode_rows(enc, &prm.b_hi, a.b_hi, C::NCP, npt, a.nkey, C::NP) ||
        !encode_rows(enc, &prm.b_lo, a.b_lo, C::NCP, npt, a.nkey, C::NP))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc::k_tcg<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tiles < a.num_sms ? tiles : a.num_sms;
    tc::k_tcg<P><<<grid, 192, C::SMEM_BYTES, s>>>(prm);
    return cudaGetLastError();
}

cudaError_t tcg_launch(int p, const TCGArgs& a, cudaStream_t s) {
    switch (p) {
        case 2: return launch_tcg<2>(a, s);
        case 3: return launch_tcg<3>(a, s);
        case 4: return launch_tcg<4>(a, s);
        case 5: return launch_tcg<5>(a, s);
        case 6: return launch_tcg<6>(a, s);
        case 7: return launch_tcg<7>(a, s);
        case 8: return launch_tcg<8>(a, s);
        case 9: return launch_tcg<9>(a, s);
        case 10: return launch_tcg<10>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t tc_launch(int p, const TCArgs& a, cudaStream_t s) {
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
