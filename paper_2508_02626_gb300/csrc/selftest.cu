// selftest.cu -- self-tests of the failure paths (the paper has no counterpart).
//
// dafmm_debug_expire_wait: one launch whose bounded mbarrier wait is made to give up, so that a
// test can check on the GPU, without any fault, that an expired wait reaches the host as
// DAFMM_ERR_TIMEOUT through dafmm_sync and that the context stays usable afterwards.
//
// The wait is the one every tensor-core kernel uses (tc::mbar_wait: it gives up after 1 s of
// %globaltimer or 2^26 polls, records its site code in the context's error flag and returns
// false).  The barrier expects one arrival and nothing arrives, so its phase 0 never
// completes and the wait runs out; the kernel then invalidates the barrier and returns.
//
// dafmm_debug_check: in a library built with DAFMM_CHECK, one launch whose index check fails on
// purpose (an index one past its stated bound, into an array that is larger still), so that a
// test can check that a failed check reaches the host as DAFMM_ERR_CHECK.
#include <cuda_runtime.h>

#include <string>

#include "api_types.h"
#include "tc_common.cuh"

namespace {

constexpr int kExpireSite = 90;  // site code the expired wait records (the kernels use 11..46)

__global__ void k_expire_wait(int* err) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = dafmm::tc::smem_u32(&bar);
    dafmm::tc::mbar_init(b, 1);
    dafmm::tc::mbar_wait(b, 0, err, kExpireSite);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
}

}  // namespace

int dafmm_debug_expire_wait(dafmm_ctx* c, void* stream) {
    if (!c) return DAFMM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) {
        k_expire_wait<<<1, 32, 0, (cudaStream_t)stream>>>(c->d_err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        c->err = std::string("DAFMM_ERR_CUDA: dafmm_debug_expire_wait: ") + cudaGetErrorString(e);
        return DAFMM_ERR_CUDA;
    }
    return DAFMM_OK;
}

// ---- dafmm_debug_check: one deliberate failure of the checked build's index check ---------------
#include "check.cuh"

namespace {
#if defined(DAFMM_CHECK)
// lane l guards entry 32 + l of a 64-entry array against the bound 32: every check fails (site
// kChkDebug, the first recorded), and every access it guards would be in bounds anyway
__global__ void k_check_probe(int* out) {
    __shared__ int s[64];
    s[threadIdx.x] = (int)threadIdx.x;
    __syncwarp();
    const int i = 32 + (int)threadIdx.x;
    int v = -1;
    if (DAFMM_IN(i, 32, dafmm::kChkDebug)) v = s[i];
    if (v >= 0) out[0] = v;  // never reached: keeps the guarded load
}
#endif
}  // namespace

int dafmm_debug_check(dafmm_ctx* c, void* stream) {
    if (!c) return DAFMM_ERR_INVALID_ARG;
#if defined(DAFMM_CHECK)
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) {
        k_check_probe<<<1, 32, 0, (cudaStream_t)stream>>>(c->d_err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        c->err = std::string("DAFMM_ERR_CUDA: dafmm_debug_check: ") + cudaGetErrorString(e);
        return DAFMM_ERR_CUDA;
    }
    return DAFMM_OK;
#else
    (void)stream;
    c->err = "unsupported option: dafmm_debug_check needs a library built with DAFMM_CHECK";
    return DAFMM_ERR_UNSUPPORTED;
#endif
}
