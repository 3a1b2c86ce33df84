// selftest.cu -- dafmm_debug_expire_wait (the paper has no counterpart): one launch whose
// bounded mbarrier wait is made to give up, so that a test can check on the GPU, without any
// fault, that an expired wait reaches the host as DAFMM_ERR_TIMEOUT through dafmm_sync and
// that the context stays usable afterwards.
//
// The wait is the one every tensor-core kernel uses (tc::mbar_wait: it gives up after 1 s of
// %globaltimer or 2^26 polls, records its site code in the context's error flag and returns
// false).  The barrier expects one arrival and nothing arrives, so its phase 0 never
// completes and the wait runs out; the kernel then invalidates the barrier and returns.
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
