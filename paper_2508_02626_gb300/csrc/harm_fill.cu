// harm_fill.cu -- the multipoles' coefficients of z exponent >= 2 from their free ones, in place
// (adaptive trees in the harmonic basis: the P2M and M2M compute the free coefficients only,
// the M2P of the W lists reads every coefficient).
#include <cuda_runtime.h>

#include "internal.h"

namespace dafmm {
namespace {

struct HarmCst {
    int c[kMaxOrder + 3];  // steps of z exponent c: [c[c], c[c + 1])
};

// The homogeneous parts of a multipole expansion are harmonic (Eq. 2, the Legendre generating
// function), so Laplace's equation gives every coefficient of z exponent >= 2 from those of
// z exponent <= 1.  One warp per FP64 row: the free coefficients staged in shared memory, the
// steps a[i] = w1 a[i1] + w2 a[i2] applied in order of increasing z exponent, each result
// written to the row as it is made.
__global__ void __launch_bounds__(128) k_harm_fill(double* __restrict__ M, int nrows, const int4* __restrict__ step,
                                                   const double2* __restrict__ w, HarmCst cst, int p, int ncp,
                                                   int nh) {
    __shared__ double sbuf[4][ncp_of(kMaxOrder)];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int row = (int)(blockIdx.x * 4 + wi);
    if (row >= nrows) return;
    double* buf = sbuf[wi];
    double* r = M + (size_t)row * ncp;
    for (int k = lane; k < nh; k += 32) {
        const int i = harm_full_index(k);
        buf[i] = r[i];
    }
    __syncwarp();
    for (int c = 2; c <= p; ++c) {
        for (int s = cst.c[c] + lane; s < cst.c[c + 1]; s += 32) {
            const int4 st = step[s];
            const double2 ww = w[s];
            const double v = fma(ww.x, buf[st.y], ww.y * buf[st.z]);
            buf[st.x] = v;
            r[st.x] = v;
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t harm_fill(int p, double* M, int nrows, const int4* step, const double2* w, const int* cst, cudaStream_t s) {
    if (nrows <= 0 || p < 2) return cudaSuccess;
    if (!step || !w || p > kMaxOrder) return cudaErrorInvalidValue;
    HarmCst hc;
    for (int c = 0; c < kMaxOrder + 3; ++c) hc.c[c] = c <= p + 1 ? cst[c] : 0;
    k_harm_fill<<<(nrows + 3) / 4, 128, 0, s>>>(M, nrows, step, w, hc, p, ncp_of(p), nharm_of(p));
    return cudaGetLastError();
}

}  // namespace dafmm
