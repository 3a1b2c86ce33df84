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
// FP32 registers, write the result -- FP64 rows, or FP32 rows in the FP32 mode of uniform
// trees -- and, when asked, its TF32 split for the next stage.  (The FP32 mode's M2L takes
// F16 hi/lo splits with power-of-two scales instead of TF32 ones; see tc_common.cuh.)
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
template <int P, bool H, bool R>
__global__ void __launch_bounds__(192, 1) k_tc(const __grid_constant__ TCParams prm) {
    using C = Cfg<P, H, R>;
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
                    const int kx = kc * C::KPC;  // first element of the chunk (128-byte aligned)
                    tma_load_5d(smem_u32(st), &prm.a_hi[it.li], fb, kx, sx, sy, sz, slab);
                    tma_load_5d(smem_u32(st + C::A_BYTES), &prm.a_lo[it.li], fb, kx, sx, sy, sz, slab);
                    tma_load_3d(smem_u32(st + 2 * C::A_BYTES), &prm.b_hi, fb, kx, it.half * C::NP, key);
                    tma_load_3d(smem_u32(st + 2 * C::A_BYTES + C::B_BYTES), &prm.b_lo, fb, kx, it.half * C::NP, key);
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
                        mma_op<H>(d, ah, bl, C::IDESC, accum);  // small cross terms first
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
            // F16 operands: each term's accumulator carries the source row's scale and the
            // matrix's scalar; the factor undoing both (one per row and term) is looked up for
            // the next term right after a term's accumulator is released, before waiting for the
            // next one
            auto factor = [&](const Terms& t) -> float {
                if constexpr (H) {
                    const int bx = prm.bx[it.li], by = prm.by[it.li], bz = prm.bz[it.li];
                    if (row >= bx * by * bz) return 0.f;
                    int sx, sy, sz, slab, key;
                    t.source(it, sx, sy, sz, slab, key);
                    const int S = prm.S[it.li];
                    sx += row % bx;
                    sy += (row / bx) % by;
                    sz += row / (bx * by);
                    if (sx < 0 || sy < 0 || sz < 0 || sx >= S || sy >= S || sz >= S) return 0.f;
                    return prm.a_inv[it.li][(size_t)slab * S * S * S + ((size_t)sz * S + sy) * S + sx] * prm.inv_c[key];
                } else {
                    return 1.f;
                }
            };
            Terms tm;
            tm.first(prm.mode, it.oct);
            bool have = tm.valid() || tm.next_valid();
            int lastbuf = -1;  // the last term's accumulator stays held until the row is out
            float f = have ? factor(tm) : 0.f;
            while (have) {
                const int buf = uses & 1;
                ok = mbar_wait(smem_u32(&acc_full[buf]), accf_ph[buf], prm.err, 31);
                if (!ok) break;
                accf_ph[buf] ^= 1u;
                fence_after_sync();
                const uint32_t tb = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::NP);
                fold_term<C::NP, H, R>(tb, f, S);
                ++uses;
                have = tm.next_valid();
                if (have) {
                    fence_before_sync();
                    mbar_arrive(smem_u32(&acc_empty[buf]));
                    f = factor(tm);
                } else {
                    lastbuf = buf;
                }
            }
            if (!ok) break;
            if (lastbuf < 0) continue;  // no term (does not occur: every work item has one)
            // the summed row back into the held accumulator, then out from there
            const uint32_t tb = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(lastbuf * C::NP);
#pragma unroll
            for (int c0 = 0; c0 < C::NP; c0 += 16) tmem_st16(tb + c0, S + c0);
            tmem_wait_st();
            const int bx = prm.bx[it.li], by = prm.by[it.li], bz = prm.bz[it.li];
            const bool valid = row < bx * by * bz;
            size_t t = 0;
            if (valid) t = (size_t)out_index(prm, it, row % bx, (row / bx) % by, row / (bx * by)) * C::NCP;
            const bool f32 = prm.out_f32 != 0;
            void* orow = f32 ? static_cast<void*>(reinterpret_cast<float*>(prm.out[it.li]) + t)
                             : static_cast<void*>(prm.out[it.li] + t);
            float* hrow = prm.out_hi[it.li] ? prm.out_hi[it.li] + t : nullptr;
            float* lrow = prm.out_lo[it.li] ? prm.out_lo[it.li] + t : nullptr;
            // L2L adds to the locals that M2L wrote
            store_row<C::NP, C::NC, C::NCP, H>(tb, valid, it.half * C::NP, prm.scale[it.li], (float)prm.scale[it.li],
                                               prm.inv_r, prm.mode == kTcL2L, f32, orow, hrow, lrow);
            fence_before_sync();
            mbar_arrive(smem_u32(&acc_empty[lastbuf]));
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

// the free coefficients (harm_full_index) of FP64 rows [nrows][ncp] into TF32 parts, rows of
// nhp values (zeros past nh)
__global__ void k_split_tf32_harm(const double* __restrict__ src, size_t nrows, int ncp, int nh, int nhp,
                                  float* __restrict__ hi, float* __restrict__ lo) {
    const size_t n = nrows * nhp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nhp;
        const int k = (int)(i % nhp);
        const double x = k < nh ? src[row * ncp + harm_full_index(k)] : 0.0;
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

// ---- F16 split with power-of-two scales -------------------------------------------------------
// x = (hi + lo) / s exactly up to the rounding of lo (about 2^-22 relative to the row maximum);
// s is a power of two that puts the largest magnitude of the row in [0.5, 1), so the halves
// stay far from their overflow and the small coefficients lose at most 2^-25 of the row
// maximum to F16 subnormals.
__device__ __forceinline__ int pow2_exponent(double mx) {
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

// v is already scaled into [-1, 1]: its FP32 rounding keeps 24 bits, more than hi + lo hold
__device__ __forceinline__ void split_half(double v, __half& h, __half& l) {
    const float f = (float)v;
    h = __float2half_rn(f);
    l = __float2half_rn(f - __half2float(h));
}

// up to 8 arrays of rows split in one launch; segment s covers global rows [first[s], first[s+1])
struct F16Segments {
    const void* src[8];  // FP64 rows, or FP32 rows when src_f32
    __half* hi[8];
    __half* lo[8];
    float* inv[8];
    int first[9];
    int nseg;
    int src_f32;
    int harm;            // take the free coefficients of the harmonic basis (harm_full_index)
};

// one warp per row of src [nrows][ncp] -> hi, lo [nrows][rowlen] halves, inv[nrows].  The work
// is FP32 throughout (an FP64 value is rounded to FP32 once: the scale is a power of two, so
// scaling commutes with that rounding, and FP32 keeps more bits than hi + lo hold); FP64
// instructions run at a small fraction of the FP32 rate on this part.
__global__ void k_split_f16_rows(F16Segments sg, int nc, int ncp, int rowlen) {
    int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= sg.first[sg.nseg]) return;
    int g = 0;
    while (g + 1 < sg.nseg && row >= sg.first[g + 1]) ++g;
    row -= sg.first[g];
    __half* __restrict__ hi = sg.hi[g];
    __half* __restrict__ lo = sg.lo[g];
    float* __restrict__ inv = sg.inv[g];
    constexpr int KMAX = 12;  // up to 32 x 12 = 384 coefficients per row (p <= 10: 286)
    float v[KMAX];
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        const int k = lane + 32 * j;
        float x = 0.f;
        if (k < nc) {
            const int kk = sg.harm ? harm_full_index(k) : k;
            x = sg.src_f32 ? static_cast<const float*>(sg.src[g])[(size_t)row * ncp + kk]
                           : (float)static_cast<const double*>(sg.src[g])[(size_t)row * ncp + kk];
        }
        v[j] = x;
        mx = fmaxf(mx, fabsf(x));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
    const float sc = ldexpf(1.f, -e);
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        const int k = lane + 32 * j;
        if (k >= rowlen) break;
        const float f = v[j] * sc;
        const __half h = __float2half_rn(f);
        hi[(size_t)row * rowlen + k] = h;
        lo[(size_t)row * rowlen + k] = __float2half_rn(f - __half2float(h));
    }
    if (lane == 0) inv[row] = ldexpf(1.f, e);
}

// per row b of the matrices: the largest magnitude over all matrices -> exponent in er[b]
__global__ void k_k16_rowexp(const double* __restrict__ K, int nkey, int nc, int ncp, int npt, float* er) {
    const int b = blockIdx.x;
    double mx = 0.0;
    if (b < nc)
        for (size_t i = threadIdx.x; i < (size_t)nkey * nc; i += blockDim.x) {
            const size_t key = i / nc, a = i % nc;
            mx = fmax(mx, fabs(K[(key * nc + b) * ncp + a]));
        }
    __shared__ double red[256];
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) er[b] = (float)pow2_exponent(red[0]);
}

// per matrix: the largest magnitude after the row scales -> exponent in ec[key]
__global__ void k_k16_keyexp(const double* __restrict__ K, int nc, int ncp, const float* __restrict__ er, float* ec) {
    const int key = blockIdx.x;
    double mx = 0.0;
    for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) {
        const int b = i / nc, a = i % nc;
        mx = fmax(mx, fabs(ldexp(K[((size_t)key * nc + b) * ncp + a], -(int)er[b])));
    }
    __shared__ double red[256];
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) ec[key] = (float)pow2_exponent(red[0]);
}

__global__ void k_k16_split(const double* __restrict__ K, int nkey, int nc, int ncp, int npt, int rowlen,
                            const float* __restrict__ er, const float* __restrict__ ec, __half* __restrict__ hi,
                            __half* __restrict__ lo, float* __restrict__ inv_r, float* __restrict__ inv_c) {
    const size_t n = (size_t)nkey * npt * rowlen;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(i % rowlen);
        const size_t rk = i / rowlen;
        const int b = (int)(rk % npt);
        const size_t key = rk / npt;
        double v = 0.0;
        if (b < nc && a < nc) v = ldexp(K[(key * nc + b) * ncp + a], -(int)er[b] - (int)ec[key]);
        __half h, l;
        split_half(v, h, l);
        hi[i] = h;
        lo[i] = l;
        if (a == 0 && key == 0) inv_r[b] = b < nc ? ldexpf(1.f, (int)er[b]) : 1.f;
        if (a == 0 && b == 0) inv_c[key] = ldexpf(1.f, (int)ec[key]);
    }
}

// K^_v in the harmonic basis (one block per matrix): rows are the free coefficients of the
// output, columns the free coefficients of the input through the expansion X [nc][nh] that
// restores every coefficient from them, Kh[key][r][j] = sum_i K[key][free r][i] X[i][j]
__global__ void k_harm_K(const double* __restrict__ K, int nc, int ncp, const double* __restrict__ X, int nh, int nhp,
                         double* __restrict__ Kh) {
    const size_t key = blockIdx.x;
    for (int e = threadIdx.x; e < nh * nhp; e += blockDim.x) {
        const int r = e / nhp, j = e % nhp;
        double acc = 0.0;
        if (j < nh) {
            const double* kr = K + (key * nc + harm_full_index(r)) * ncp;
            for (int i = 0; i < nc; ++i) acc = fma(kr[i], X[(size_t)i * nh + j], acc);
        }
        Kh[(key * nh + r) * nhp + j] = acc;
    }
}

// rows of free coefficients (FP32, stride nhp) -> full expansion rows (FP32 or FP64, stride ncp),
// one warp per row: the free coefficients go to their places, then the others follow from
// Laplace's equation in order of increasing z exponent (each step a[i] = w1 a[i1] + w2 a[i2]
// reads two coefficients of z exponent c - 2), columns nc..ncp-1 are zeros; optionally the TF32
// split of the written row
struct HarmSegments {
    const float* red[kTcMaxLevels];
    void* full[kTcMaxLevels];
    float* hi[kTcMaxLevels];
    float* lo[kTcMaxLevels];
    int first[kTcMaxLevels + 1];
    int nseg;
    int full_f32;
    int cst[kMaxOrder + 3];  // steps of z exponent c: [cst[c], cst[c + 1]), c = 2..p
};

__global__ void __launch_bounds__(128) k_harm_expand(HarmSegments sg, const int4* __restrict__ step,
                                                     const float2* __restrict__ w, int p, int nc, int ncp, int nh,
                                                     int nhp) {
    __shared__ float sbuf[4][ncp_of(kMaxOrder)];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    int row = (int)(blockIdx.x * 4 + wi);
    if (row >= sg.first[sg.nseg]) return;
    int g = 0;
    while (g + 1 < sg.nseg && row >= sg.first[g + 1]) ++g;
    row -= sg.first[g];
    float* buf = sbuf[wi];
    const float* r = sg.red[g] + (size_t)row * nhp;
    for (int k = lane; k < nh; k += 32) buf[harm_full_index(k)] = r[k];
    __syncwarp();
    for (int c = 2; c <= p; ++c) {
        for (int s = sg.cst[c] + lane; s < sg.cst[c + 1]; s += 32) {
            const int4 st = step[s];
            const float2 ww = w[s];
            buf[st.x] = fmaf(ww.x, buf[st.y], ww.y * buf[st.z]);
        }
        __syncwarp();
    }
    float* hi = sg.hi[g] ? sg.hi[g] + (size_t)row * ncp : nullptr;
    float* lo = sg.lo[g] ? sg.lo[g] + (size_t)row * ncp : nullptr;
    for (int k = lane; k < ncp; k += 32) {
        const float v = k < nc ? buf[k] : 0.f;
        if (sg.full_f32) static_cast<float*>(sg.full[g])[(size_t)row * ncp + k] = v;
        else static_cast<double*>(sg.full[g])[(size_t)row * ncp + k] = (double)v;
        if (hi) {
            const float h = to_tf32(v);
            hi[k] = h;
            lo[k] = to_tf32(v - h);
        }
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

int tc_rowlen16(int p) { return (ncoef_of(p) + 15) / 16 * 16; }

int tc_npt_h(int p) {
    const int npf = (nharm_of(p) + 15) / 16 * 16;
    if (npf <= 192) return npf;
    return 2 * ((npf / 2 + 15) / 16 * 16);
}

int tc_rowlen16h(int p) { return (nharm_of(p) + 15) / 16 * 16; }

cudaError_t tc_split_f16_multi(int nseg, const void* const* src, const int* nrows, void* const* hi, void* const* lo,
                               float* const* inv, int p, cudaStream_t s, bool src_f32, bool harm) {
    if (nseg < 1 || nseg > 8) return cudaErrorInvalidValue;
    if (ncoef_of(p) > 32 * 12) return cudaErrorInvalidValue;
    tc::F16Segments sg;
    memset(&sg, 0, sizeof(sg));
    sg.nseg = nseg;
    sg.src_f32 = src_f32 ? 1 : 0;
    sg.harm = harm ? 1 : 0;
    for (int g = 0; g < nseg; ++g) {
        sg.src[g] = src[g];
        sg.hi[g] = static_cast<__half*>(hi[g]);
        sg.lo[g] = static_cast<__half*>(lo[g]);
        sg.inv[g] = inv[g];
        sg.first[g + 1] = sg.first[g] + nrows[g];
    }
    const int total = sg.first[nseg];
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(((size_t)total * 32 + 255) / 256);
    tc::k_split_f16_rows<<<blocks, 256, 0, s>>>(sg, harm ? nharm_of(p) : ncoef_of(p), ncp_of(p),
                                                 harm ? tc_rowlen16h(p) : tc_rowlen16(p));
    return cudaGetLastError();
}

cudaError_t tc_split_f16(const double* src, int nrows, int p, void* hi, void* lo, float* inv, cudaStream_t s) {
    const void* sv = src;
    return tc_split_f16_multi(1, &sv, &nrows, &hi, &lo, &inv, p, s, false, false);
}

cudaError_t tc_prepare_k16(const double* K, int nkey, int p, void* hi, void* lo, float* inv_r, float* inv_c,
                           float* scratch, cudaStream_t s) {
    const int nc = ncoef_of(p), ncp = ncp_of(p), npt = tc_npt(p), rowlen = tc_rowlen16(p);
    float* er = scratch;        // npt row exponents
    float* ec = scratch + npt;  // nkey matrix exponents
    tc::k_k16_rowexp<<<npt, 256, 0, s>>>(K, nkey, nc, ncp, npt, er);
    tc::k_k16_keyexp<<<nkey, 256, 0, s>>>(K, nc, ncp, er, ec);
    tc::k_k16_split<<<152 * 16, 256, 0, s>>>(K, nkey, nc, ncp, npt, rowlen, er, ec, static_cast<__half*>(hi),
                                              static_cast<__half*>(lo), inv_r, inv_c);
    return cudaGetLastError();
}

cudaError_t tc_prepare_k16h(const double* K, int nkey, int p, const double* X, double* Kh, void* hi, void* lo,
                            float* inv_r, float* inv_c, float* scratch, float* thi, float* tlo, cudaStream_t s) {
    const int nc = ncoef_of(p), ncp = ncp_of(p), nh = nharm_of(p), nhp = (nh + 7) / 8 * 8;
    const int npt = tc_npt_h(p), rowlen = tc_rowlen16h(p);
    float* er = scratch;        // npt row exponents
    float* ec = scratch + npt;  // nkey matrix exponents
    tc::k_harm_K<<<nkey, 256, 0, s>>>(K, nc, ncp, X, nh, nhp, Kh);
    tc::k_k16_rowexp<<<npt, 256, 0, s>>>(Kh, nkey, nh, nhp, npt, er);
    tc::k_k16_keyexp<<<nkey, 256, 0, s>>>(Kh, nh, nhp, er, ec);
    tc::k_k16_split<<<152 * 16, 256, 0, s>>>(Kh, nkey, nh, nhp, npt, rowlen, er, ec, static_cast<__half*>(hi),
                                              static_cast<__half*>(lo), inv_r, inv_c);
    tc::k_split_rows<<<152 * 16, 256, 0, s>>>(Kh, nkey, nh, nhp, npt, thi, tlo);
    return cudaGetLastError();
}

cudaError_t tc_harm_expand(int p, int nseg, const float* const* red, void* const* full, float* const* hi,
                           float* const* lo, const int* nrows, bool full_f32, const int4* step, const float2* w,
                           const int* cst, cudaStream_t s) {
    if (nseg < 1 || nseg > kTcMaxLevels) return cudaErrorInvalidValue;
    tc::HarmSegments sg;
    memset(&sg, 0, sizeof(sg));
    sg.nseg = nseg;
    sg.full_f32 = full_f32 ? 1 : 0;
    for (int g = 0; g < nseg; ++g) {
        sg.red[g] = red[g];
        sg.full[g] = full[g];
        sg.hi[g] = hi ? hi[g] : nullptr;
        sg.lo[g] = lo ? lo[g] : nullptr;
        sg.first[g + 1] = sg.first[g] + nrows[g];
    }
    for (int c = 0; c <= p + 1; ++c) sg.cst[c] = cst[c];
    const int total = sg.first[nseg];
    if (total == 0) return cudaSuccess;
    const int nh = nharm_of(p);
    tc::k_harm_expand<<<(total + 3) / 4, 128, 0, s>>>(sg, step, w, p, ncoef_of(p), ncp_of(p), nh, (nh + 7) / 8 * 8);
    return cudaGetLastError();
}

cudaError_t tc_split_tf32(const double* src, float* hi, float* lo, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    tc::k_split_tf32<<<blocks, 256, 0, s>>>(src, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t tc_split_tf32_harm(const double* src, size_t nrows, int p, float* hi, float* lo, cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    const int nh = nharm_of(p), nhp = harm_row(p);
    const unsigned blocks = (unsigned)std::min<size_t>((nrows * nhp + 255) / 256, 152 * 16);
    tc::k_split_tf32_harm<<<blocks, 256, 0, s>>>(src, nrows, ncp_of(p), nh, nhp, hi, lo);
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
static bool encode_level(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const void* base, int rowlen, int S,
                         int bx, int by, int bz, bool f16) {
    const cuuint64_t esz = f16 ? 2 : 4;
    const cuuint64_t dims[5] = {(cuuint64_t)rowlen, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)S, 8};
    const cuuint64_t row = (cuuint64_t)rowlen * esz;
    const cuuint64_t strides[4] = {row, row * S, row * S * S, row * S * S * S};
    const cuuint32_t box[5] = {(cuuint32_t)(128 / esz), (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base),
               dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int P, bool H, bool R = false>
static cudaError_t launch_tc(const TCArgs& a, cudaStream_t s) {
    using C = tc::Cfg<P, H, R>;
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    TCParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.mode = a.mode;
    prm.nhalf = C::NHALF;
    prm.out_f32 = a.out_f32 ? 1 : 0;
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
        prm.a_inv[li] = a.a_inv[src];
        if (!encode_level(enc, &prm.a_hi[li], a.a_hi[src], C::ROWLEN, S, bx, by, bz, H) ||
            !encode_level(enc, &prm.a_lo[li], a.a_lo[src], C::ROWLEN, S, bx, by, bz, H))
            return cudaErrorInvalidValue;
    }
    prm.tile_base[prm.nlev] = tiles;
    prm.ntiles = tiles;
    const int npt = C::NPT;
    prm.inv_r = a.inv_r;
    prm.inv_c = a.inv_c;
    if (!encode_rows(enc, &prm.b_hi, a.b_hi, C::ROWLEN, npt, a.nkey, C::NPL, H) ||
        !encode_rows(enc, &prm.b_lo, a.b_lo, C::ROWLEN, npt, a.nkey, C::NPL, H))
        return cudaErrorInvalidValue;
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc::k_tc<P, H, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tiles < a.num_sms ? tiles : a.num_sms;
    tc::k_tc<P, H, R><<<grid, 192, C::SMEM_BYTES, s>>>(prm);
    return cudaGetLastError();
}
template <int P>
static cudaError_t launch_tc_any(const TCArgs& a, cudaStream_t s) {
    if (a.f16) {
        if (a.mode != kTcM2L) return cudaErrorInvalidValue;
        return a.harm ? launch_tc<P, true, true>(a, s) : launch_tc<P, true, false>(a, s);
    }
    if (a.harm) return a.mode == kTcM2L ? launch_tc<P, false, true>(a, s) : cudaErrorInvalidValue;
    return launch_tc<P, false>(a, s);
}

cudaError_t tc_launch(int p, const TCArgs& a, cudaStream_t s) {
    switch (p) {
        case 2: return launch_tc_any<2>(a, s);
        case 3: return launch_tc_any<3>(a, s);
        case 4: return launch_tc_any<4>(a, s);
        case 5: return launch_tc_any<5>(a, s);
        case 6: return launch_tc_any<6>(a, s);
        case 7: return launch_tc_any<7>(a, s);
        case 8: return launch_tc_any<8>(a, s);
        case 9: return launch_tc_any<9>(a, s);
        case 10: return launch_tc_any<10>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dafmm
