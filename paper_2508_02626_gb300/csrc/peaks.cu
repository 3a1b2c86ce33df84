// peaks.cu -- dafmm_probe_peak (the paper has no counterpart): the unit rates of this GPU that
// the rooflines of the non-HBM, non-BF16 kernels divide by, measured instead of derived from
// unit counts and clocks.
//
//   DAFMM_PEAK_FFMA      scalar FP32 FMA          2 flops per instruction and lane
//   DAFMM_PEAK_FFMA2     packed FP32x2 FMA        4 flops per instruction and lane
//   DAFMM_PEAK_DFMA      FP64 FMA                 2 flops per instruction and lane
//   DAFMM_PEAK_RSQRT     rsqrt.approx.ftz.f32     1 result per instruction and lane
//   DAFMM_PEAK_MMA_TF32  tcgen05.mma kind::tf32   M=128 N=256 K=8: 2*128*256*8 flops each
//   DAFMM_PEAK_MMA_F16   tcgen05.mma kind::f16    M=128 N=256 K=16: 2*128*256*16 flops each
//
// The ALU probes run 16 independent dependency chains per thread (enough to cover the pipe
// latencies) in 8 blocks of 256 threads per SM; the result is kept alive by a conditional
// store that never happens.  The MMA probe runs one CTA per SM (its shared-memory request
// admits no second one, so the TMEM allocation of 512 columns never waits): one thread issues
// back-to-back MMAs from shared-memory operands into two TMEM accumulators in turn, commits
// them to an mbarrier and waits for it with the bounded wait of the tensor-core kernels (on
// expiry the probe returns DAFMM_ERR_TIMEOUT).  Each probe is launched once to warm up, then
// timed with CUDA events around one launch of about 20-100 ms.
#include <cuda_runtime.h>

#include <string>

#include "api_types.h"
#include "tc_common.cuh"

namespace {

using namespace dafmm::tc;

__device__ int g_probe_err;
__device__ float g_probe_sink;

__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__global__ void __launch_bounds__(256) k_alu_probe(int iters, float seed) {
    constexpr int C = 16;
    const float t = seed + 1e-6f * (float)threadIdx.x;
    if constexpr (KIND == DAFMM_PEAK_DFMA) {
        double a[C];
#pragma unroll
        for (int j = 0; j < C; ++j) a[j] = (double)t + 1e-3 * j;
        const double b = 0.999999, c = 1e-7;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < C; ++j) a[j] = fma(a[j], b, c);
        }
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < C; ++j) s += a[j];
        if (s == 123.25) g_probe_sink = (float)s;
    } else if constexpr (KIND == DAFMM_PEAK_FFMA2) {
        float2 a[C / 2];
#pragma unroll
        for (int j = 0; j < C / 2; ++j) a[j] = make_float2(t + 1e-3f * j, t - 1e-3f * j);
        const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < C / 2; ++j) a[j] = __ffma2_rn(a[j], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < C / 2; ++j) s += a[j].x + a[j].y;
        if (s == 123.25f) g_probe_sink = s;
    } else {
        float a[C];
#pragma unroll
        for (int j = 0; j < C; ++j) a[j] = t + 1e-3f * j + 0.5f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if constexpr (KIND == DAFMM_PEAK_RSQRT) a[j] = rsqrt_fast(a[j]);
                else a[j] = fmaf(a[j], 0.999999f, 1e-7f);
            }
        }
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < C; ++j) s += a[j];
        if (s == 123.25f) g_probe_sink = s;
    }
}

constexpr int kMmaN = 256;
constexpr int kAbytes = 128 * 128;        // 128 rows x one 128-byte K chunk
constexpr int kBbytes = kMmaN * 128;      // 256 rows x one 128-byte K chunk
constexpr int kMmaSmem = 120 * 1024;      // > half of the SM's shared memory: one CTA per SM
constexpr int kProbeSite = 91;            // site code of an expired wait of this probe

template <bool F16>
__global__ void __launch_bounds__(128, 1) k_mma_probe(int reps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* A = base;
    unsigned char* Bm = base + kAbytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Bm + kBbytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    // operands: small finite values (F16 ones or TF32 ones, per the kind)
    for (int i = threadIdx.x; i < (kAbytes + kBbytes) / 4; i += blockDim.x) {
        const float v = 0.25f + 0.125f * (float)(i & 7);
        uint32_t w;
        if constexpr (F16) {
            const __half h = __float2half_rn(v);
            const uint16_t u = *reinterpret_cast<const uint16_t*>(&h);
            w = (uint32_t)u | ((uint32_t)u << 16);
        } else {
            w = __float_as_uint(v);
        }
        reinterpret_cast<uint32_t*>(A)[i] = w;  // A and B are contiguous
    }
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor core
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        const uint64_t ad = smem_desc_sw128(smem_u32(A)), bd = smem_desc_sw128(smem_u32(Bm));
        const uint32_t id = F16 ? idesc_f16(128, kMmaN) : idesc_tf32(128, kMmaN);
        for (int r = 0; r < reps; ++r) {
            const uint32_t d = tmem + (uint32_t)((r & 1) * kMmaN);
#pragma unroll
            for (int k = 0; k < 4; ++k)  // the four 32-byte K steps of the chunk
                mma_op<F16>(d, ad + 2 * k, bd + 2 * k, id, (r > 1 || k > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(bar));
        mbar_wait(smem_u32(bar), 0, &g_probe_err, kProbeSite);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int KIND>
cudaError_t launch_probe(int sms, long long work, cudaStream_t s) {
    if constexpr (KIND == DAFMM_PEAK_MMA_TF32 || KIND == DAFMM_PEAK_MMA_F16) {
        constexpr bool F16 = KIND == DAFMM_PEAK_MMA_F16;
        cudaError_t e = cudaFuncSetAttribute(k_mma_probe<F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
        if (e != cudaSuccess) return e;
        k_mma_probe<F16><<<sms, 128, kMmaSmem, s>>>((int)work);
    } else {
        k_alu_probe<KIND><<<sms * 8, 256, 0, s>>>((int)work, 0.25f);
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" int dafmm_probe_peak(int device, int kind, double* rate, double* ms) {
    if (!rate || kind < DAFMM_PEAK_FFMA || kind > DAFMM_PEAK_MMA_F16) return DAFMM_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DAFMM_ERR_INVALID_ARG;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return DAFMM_ERR_CUDA;
    // work per launch (iterations of the 16-chain loop, or MMA pairs of K chunks) sized for
    // about 20-100 ms at the nominal rates of a GB300
    long long work = 0;
    double ops_per_unit = 0.0;  // counted operations per unit of work, whole grid
    const double lanes = (double)sms * 8 * 256;
    switch (kind) {
        case DAFMM_PEAK_FFMA: work = 200000; ops_per_unit = lanes * 16 * 2; break;
        case DAFMM_PEAK_FFMA2: work = 200000; ops_per_unit = lanes * 8 * 4; break;
        case DAFMM_PEAK_DFMA: work = 4000; ops_per_unit = lanes * 16 * 2; break;
        case DAFMM_PEAK_RSQRT: work = 40000; ops_per_unit = lanes * 16; break;
        case DAFMM_PEAK_MMA_TF32: work = 200000; ops_per_unit = (double)sms * 4 * 2.0 * 128 * kMmaN * 8; break;
        case DAFMM_PEAK_MMA_F16: work = 200000; ops_per_unit = (double)sms * 4 * 2.0 * 128 * kMmaN * 16; break;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int zero = 0;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_probe_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    auto run = [&](long long w) -> cudaError_t {
        switch (kind) {
            case DAFMM_PEAK_FFMA: return launch_probe<DAFMM_PEAK_FFMA>(sms, w, s);
            case DAFMM_PEAK_FFMA2: return launch_probe<DAFMM_PEAK_FFMA2>(sms, w, s);
            case DAFMM_PEAK_DFMA: return launch_probe<DAFMM_PEAK_DFMA>(sms, w, s);
            case DAFMM_PEAK_RSQRT: return launch_probe<DAFMM_PEAK_RSQRT>(sms, w, s);
            case DAFMM_PEAK_MMA_TF32: return launch_probe<DAFMM_PEAK_MMA_TF32>(sms, w, s);
            default: return launch_probe<DAFMM_PEAK_MMA_F16>(sms, w, s);
        }
    };
    float t = 0.f;
    if (e == cudaSuccess) e = run(work / 10);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = run(work);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&err, g_probe_err, sizeof(int));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return DAFMM_ERR_CUDA;
    if (err) return DAFMM_ERR_TIMEOUT;
    *rate = ops_per_unit * (double)work / ((double)t * 1e-3);
    if (ms) *ms = t;
    return DAFMM_OK;
}
