// tc_gather.cu -- the M2L contraction (Eq. 5) of adaptive trees and forests on the tensor
// cores (tcgen05, sm_103a).  The targets of one work item are 128 boxes of one level and
// octant (a group of `tg`); for each of the 189 displacement terms the source box of every
// target is found through its parent's colleague table, and the source rows are gathered
// into shared memory (the uniform-tree kernel in tc_ops.cu loads them as one TMA box).
#include "check.cuh"
#include "tc_common.cuh"

namespace dafmm {
namespace tc {

// ---- gathered M2L: adaptive trees and forests ---------------------------------------------------
// Same pipeline as k_tc, but the A rows (source multipoles) of a 128-target tile are gathered
// one 16-byte chunk at a time with cp.async into the 128-byte-swizzled K-major layout that a
// TMA box would produce (chunk j of row r at (r / 8) * 1024 + (r % 8) * 128 + (j ^ r % 8) * 16),
// zero-filled for missing sources and for columns past ncp.  Two producer warps gather, half the
// rows each (one warp issuing all of a stage's copies paced the kernel); lane 0 of the first
// also loads the K^_v tile by TMA.  A stage is signalled full once the TMA bytes have landed and
// every producer lane has seen its own copies complete, fenced them for the async proxy and
// arrived (65 arrivals: 2 x 32 lanes + the expect_tx arrival).
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

// the source of a target for the displacement term `tm` is its parent's colleague at offset
// a (slot) and that box's child sc, with o - v = 2a + sc
__device__ __forceinline__ void term_slot(const Terms& tm, int& slot, int& sc) {
    sc = 0;
    slot = 0;
    for (int d = 0; d < 3; ++d) {
        const int dd = tm.o[d] - tm.v[d];
        const int c = dd & 1;
        const int a = (dd - c) >> 1;
        sc |= c << d;
        slot = slot * 3 + (a + 1);
    }
}
// the two dependent loads of that lookup, for a target whose parent is `par` (-1: none)
__device__ __forceinline__ int colleague_of(const TCGParams& prm, int par, int slot) {
    return par >= 0 && DAFMM_IN(par, prm.nbox, kChkGatherSource) ? prm.colleague[27 * par + slot] : -1;
}
__device__ __forceinline__ int child_of(const TCGParams& prm, int Q, int sc) {
    const int s = Q >= 0 && DAFMM_IN(Q, prm.nbox, kChkGatherSource) ? prm.child[8 * Q + sc] : -1;
    return s < 0 || DAFMM_IN(s, prm.nbox, kChkGatherSource) ? s : -1;
}
__device__ __forceinline__ int term_key(const Terms& tm) {
    return (tm.v[0] + 3) * 49 + (tm.v[1] + 3) * 7 + (tm.v[2] + 3);
}

// gather warps: warp 0 (and the TMA of the matrices) takes rows 0-63 of every stage, warp 6
// rows 64-127
constexpr int kTcgThreads = 224;

template <int P, bool H, bool R>
__global__ void __launch_bounds__(kTcgThreads, 1) k_tcg(const __grid_constant__ TCGParams prm) {
    using C = Cfg<P, H, R>;
    constexpr int ESZ = H ? 2 : 4;  // operand element bytes
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* bar_area = base + C::STAGES * C::STAGE_BYTES + C::SLACK;
    uint64_t* full = reinterpret_cast<uint64_t*>(bar_area);
    uint64_t* empty = full + C::STAGES;
    uint64_t* acc_full = empty + C::STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 65);  // 2 x 32 gather lanes + the expect_tx arrival
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

    if (warp == 0 || warp == 6) {
        // ------- gather producers (two whole warps, half the rows each) + TMA of the matrices -------
        const int pw = warp == 0 ? 0 : 1;  // rows 64 pw .. 64 pw + 63
        if (warp == 0 && lane == 0) {
            prefetch_map(&prm.b_hi);
            prefetch_map(&prm.b_lo);
        }
        int stage = 0;
        uint32_t phase = 0;
        // the stage whose copies are committed but not yet signalled: it is signalled once the
        // next stage's copies are issued (holding more stages back starves the MMAs while this
        // warp issues)
        int pend = -1;
        int armed[C::STAGES];
        for (int s = 0; s < C::STAGES; ++s) armed[s] = -1;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const GItem it = gdecode(prm, w);
            const int start = prm.grp_start[it.g] + it.tile * 128;
            const int cnt = min(128, prm.grp_count[it.g] - it.tile * 128);
            int par[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = lane + 32 * (i + 2 * pw);
                const int t = r < cnt ? prm.tg[start + r] : -1;
                par[i] = t >= 0 && DAFMM_IN(t, prm.nbox, kChkGatherSource) ? prm.parent[t] : -1;
            }
            // the valid terms in order, the source lookups running ahead: while the rows of a
            // term are gathered, the children of the next term's colleagues and the colleagues
            // of the term after it are being loaded
            Terms tm;
            tm.first(kTcM2L, prm.grp_oct[it.g]);
            bool have = tm.valid() || tm.next_valid();
            int src[2], qn[2];
            int slot, sc;
            term_slot(tm, slot, sc);
#pragma unroll
            for (int i = 0; i < 2; ++i) src[i] = child_of(prm, colleague_of(prm, par[i], slot), sc);
            Terms tn = tm;
            bool hn = have && tn.next_valid();
            if (hn) term_slot(tn, slot, sc);
#pragma unroll
            for (int i = 0; i < 2; ++i) qn[i] = hn ? colleague_of(prm, par[i], slot) : -1;
            while (have && ok) {
                int srcn[2], qnn[2];
                if (hn) term_slot(tn, slot, sc);
#pragma unroll
                for (int i = 0; i < 2; ++i) srcn[i] = hn ? child_of(prm, qn[i], sc) : -1;
                Terms tnn = tn;
                const bool hnn = hn && tnn.next_valid();
                if (hnn) term_slot(tnn, slot, sc);
#pragma unroll
                for (int i = 0; i < 2; ++i) qnn[i] = hnn ? colleague_of(prm, par[i], slot) : -1;
                const int key = term_key(tm);
                for (int kc = 0; kc < C::NKC; ++kc) {
                    int got = 1;
                    if (lane == 0) got = mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, prm.err, 41) ? 1 : 0;
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (!got) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = base + stage * C::STAGE_BYTES;
                    if (warp == 0 && lane == 0) {
                        const uint32_t fb = smem_u32(&full[stage]);
                        mbar_expect_tx(fb, 2u * C::B_BYTES);
                        armed[stage] = (int)phase;
                        tma_load_3d(smem_u32(st + 2 * C::A_BYTES), &prm.b_hi, fb, kc * C::KPC, it.half * C::NP, key);
                        tma_load_3d(smem_u32(st + 2 * C::A_BYTES + C::B_BYTES), &prm.b_lo, fb, kc * C::KPC,
                                    it.half * C::NP, key);
                    }
                    const uint32_t sa = smem_u32(st);
                    const char* ahi = static_cast<const char*>(prm.a_hi);
                    const char* alo = static_cast<const char*>(prm.a_lo);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int r = lane + 32 * (i + 2 * pw);
                        const size_t rowoff = src[i] >= 0 ? (size_t)src[i] * C::ROWLEN : 0;
                        const uint32_t rbase = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = kc * C::KPC + j * (16 / ESZ);  // first element of the 16-byte chunk
                            const bool hv = src[i] >= 0 && col < C::ROWLEN;
                            const size_t e = hv ? (rowoff + col) * ESZ : 0;
                            const uint32_t off = rbase + (uint32_t)(((j ^ (r & 7)) & 7) << 4);
                            cp_async16(sa + off, ahi + e, hv ? 16u : 0u);
                            cp_async16(sa + C::A_BYTES + off, alo + e, hv ? 16u : 0u);
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
                tm = tn;
                tn = tnn;
                have = hn;
                hn = hnn;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    src[i] = srcn[i];
                    qn[i] = qnn[i];
                }
            }
        }
        if (pend >= 0) {
            cp_async_wait<0>();
            fence_proxy_async_smem();
            mbar_arrive(smem_u32(&full[pend]));
        }
        // every copy this warp armed must have landed before the block may exit
        if (warp == 0 && lane == 0)
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
                        mma_op<H>(d, ah, bl, C::IDESC, accum);
                        accum = 1;
                        mma_op<H>(d, al, bh, C::IDESC, 1);
                        mma_op<H>(d, ah, bh, C::IDESC, 1);
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
    } else if (warp >= 2 && warp <= 5) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;
        const int row = 32 * q + lane;
        uint32_t accf_ph[2] = {0, 0};
        int uses = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < prm.ntiles && ok; w += gridDim.x) {
            const GItem it = gdecode(prm, w);
            const int cnt = min(128, prm.grp_count[it.g] - it.tile * 128);
            int trow = row < cnt ? prm.tg[prm.grp_start[it.g] + it.tile * 128 + row] : -1;
            if (trow >= 0 && !DAFMM_IN(trow, prm.nbox, kChkGatherSource)) trow = -1;
            const int tpar = trow >= 0 ? prm.parent[trow] : -1;
            float S[C::NP];
#pragma unroll
            for (int j = 0; j < C::NP; ++j) S[j] = 0.f;
            // F16 operands: the factor undoing the source row's scale and the matrix's scalar,
            // looked up for the next term before waiting for its accumulator
            auto factor = [&](const Terms& t) -> float {
                if constexpr (H) {
                    int slot, sc;
                    term_slot(t, slot, sc);
                    const int sb = child_of(prm, colleague_of(prm, tpar, slot), sc);
                    return sb >= 0 ? prm.a_inv[sb] * prm.inv_c[term_key(t)] : 0.f;
                } else {
                    return 1.f;
                }
            };
            Terms tm;
            tm.first(kTcM2L, prm.grp_oct[it.g]);
            bool have = tm.valid() || tm.next_valid();
            float f = have ? factor(tm) : 0.f;
            while (have) {
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_full[buf]), accf_ph[buf], prm.err, 46);
                if (!ok) break;
                accf_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t tb = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::NP);
                fold_term<C::NP, H, R>(tb, f, S);
                fence_before_sync();
                mbar_arrive(smem_u32(&acc_empty[buf]));
                ++uses;
                have = tm.next_valid();
                if (have) f = factor(tm);
            }
            if (!ok) break;
            if (trow >= 0) {
                // FP64 rows; in the harmonic basis FP32 rows of the free coefficients (expanded
                // afterwards)
                double* orow = prm.out + (size_t)trow * C::NCP;
                float* orowf = reinterpret_cast<float*>(prm.out) + (size_t)trow * C::NCP;
                const double sc = 1.0 / prm.geom[trow].w;
#pragma unroll
                for (int j = 0; j < C::NP; ++j) {
                    const int b = it.half * C::NP + j;
                    double v = 0.0;
                    if (b < C::NC) {
                        v = (double)S[j] * sc;
                        if constexpr (H) v *= (double)prm.inv_r[b];
                    }
                    if (b < C::NCP) {
                        if constexpr (R) orowf[b] = (float)v;
                        else orow[b] = v;
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
}  // namespace tc

template <int P, bool H, bool R = false>
static cudaError_t launch_tcg(const TCGArgs& a, cudaStream_t s) {
    using C = tc::Cfg<P, H, R>;
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    if (a.ngroups > kTcgMaxGroups) return cudaErrorInvalidValue;
    TCGParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.a_hi = a.a_hi;
    prm.a_lo = a.a_lo;
    prm.a_inv = a.a_inv;
    prm.inv_r = a.inv_r;
    prm.inv_c = a.inv_c;
    prm.tg = a.tg;
    prm.parent = a.parent;
    prm.colleague = a.colleague;
    prm.child = a.child;
    prm.geom = a.geom;
    prm.out = a.out;
    prm.nhalf = C::NHALF;
    prm.err = a.err;
#if defined(DAFMM_CHECK)
    prm.nbox = a.nbox;
#endif
    int tiles = 0, ng = 0;
    for (int o = 0; o < 8; ++o)
        for (int g = 0; g < a.ngroups; ++g) {
            // only non-empty groups (the decode relies on it)
            if (a.grp_oct[g] != o || a.grp_count[g] <= 0) continue;
            prm.grp_start[ng] = a.grp_start[g];
            prm.grp_count[ng] = a.grp_count[g];
            prm.grp_oct[ng] = o;
            prm.tile_base[ng] = tiles;
            tiles += (a.grp_count[g] + 127) / 128 * C::NHALF;
            ++ng;
        }
    prm.tile_base[ng] = tiles;
    prm.ngroups = ng;
    prm.ntiles = tiles;
    if (tiles == 0) return cudaSuccess;
    const int npt = C::NPT;
    if (!encode_rows(enc, &prm.b_hi, a.b_hi, C::ROWLEN, npt, a.nkey, C::NPL, H) ||
        !encode_rows(enc, &prm.b_lo, a.b_lo, C::ROWLEN, npt, a.nkey, C::NPL, H))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc::k_tcg<P, H, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tiles < a.num_sms ? tiles : a.num_sms;
    tc::k_tcg<P, H, R><<<grid, tc::kTcgThreads, C::SMEM_BYTES, s>>>(prm);
    return cudaGetLastError();
}

template <int P>
static cudaError_t launch_tcg_any(const TCGArgs& a, cudaStream_t s) {
    if (a.harm) return a.f16 ? launch_tcg<P, true, true>(a, s) : launch_tcg<P, false, true>(a, s);
    return a.f16 ? launch_tcg<P, true>(a, s) : launch_tcg<P, false>(a, s);
}

cudaError_t tcg_launch(int p, const TCGArgs& a, cudaStream_t s) {
    switch (p) {
        case 2: return launch_tcg_any<2>(a, s);
        case 3: return launch_tcg_any<3>(a, s);
        case 4: return launch_tcg_any<4>(a, s);
        case 5: return launch_tcg_any<5>(a, s);
        case 6: return launch_tcg_any<6>(a, s);
        case 7: return launch_tcg_any<7>(a, s);
        case 8: return launch_tcg_any<8>(a, s);
        case 9: return launch_tcg_any<9>(a, s);
        case 10: return launch_tcg_any<10>(a, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace dafmm
