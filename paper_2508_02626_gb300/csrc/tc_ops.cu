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
#include "tc_common.cuh"
#include "tree_common.cuh"

namespace dafmm {
namespace tc {

// ---- work items and their terms ---------------------------------------------------------------

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

// ---- the kernel -----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(192, 1) k_tc(const __grid_constant__ TCParams prm) {
    using C = Cfg<P>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage ring, then barriers
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

// ---- split of FP64 data into TF32 high/low parts ----------------------------------------------
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
    if (!encode_rows(enc, &prm.b_hi, a.b_hi, C::NCP, npt, a.nkey, C::NPL) ||
        !encode_rows(enc, &prm.b_lo, a.b_lo, C::NCP, npt, a.nkey, C::NPL))
        return cudaErrorInvalidValue;
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc::k_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tiles < a.num_sms ? tiles : a.num_sms;
    tc::k_tc<P><<<grid, 192, C::SMEM_BYTES, s>>>(prm);
    return cudaGetLastError();
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
