// da_numeric.cu -- the FMM operators of Sec. 2 evaluated with numerical DA on the GPU: the
// truncated power series arithmetic of Appendix A (products truncated at order p, powers by
// the binomial series, composition with a map, evaluation), applied step by step as a DA
// library applies it.  This is the baseline the paper's generated operators replace (Sec. 3,
// Tables 2-8 compare the two on a CPU); here both run on the same GPU, so the ratio of their
// costs can be measured on one device.  FP64 throughout.
//
// One warp per operator instance.  Its DA vectors (three variables, coefficients in the
// graded order of da_index) live in shared memory; a truncated product gives each lane
// whole output coefficients, each the sum over the pairs (i, j) of input coefficients whose
// exponents add up to its own (the order's product table).  Operators, in the variables of
// the single-operator entry points (boxes of width 1):
//   P2M  Eq. 2   q (1 + abar)^(-1/2),  abar = -2 s.d + s^2 d^2
//   P2L  Eq. 6   q (|w|^2 + abar)^(-1/2),  abar = 2 w.d' + d'^2
//   L2P  Sec. 3.2  the local polynomial and its gradient at x (DA evaluation)
//   M2P  Sec. 3.2  |d| M(d), d = s / |s|^2, and its gradient in s, in first-order DA
//   M2M  Eq. 3-4  sqrt(R) (M o M1), M1: d = (d' + d'^2 r0) R, R = 1/(1 + r0^2 d'^2 + 2 r0.d'),
//                 r0 = 1/2 - octant (child width 1), then scaled to the parent width 2
//   L2L  Eq. 7   L o M3, M3: d = r0 + d', r0 = (octant - 1/2) / 2 (parent width 1), then
//                 scaled to the child width 1/2
//   M2L  Eq. 5   sqrt(R) (M o M2), M2: d = (r0 + d') R, R = 1/|r0 + d'|^2, r0 = the
//                 displacement (target - source) in box widths
#include <cuda_runtime.h>

#include "api_types.h"
#include "da_common.cuh"
#include "internal.h"

namespace dafmm {
namespace {

constexpr int kDaVecs = 16;  // DA vectors per warp (the M2L and M2M steps use 16)

struct DaTab {
    int p, nc;
    const int* rowptr;     // product table: output k sums a[pairs[e].x] * b[pairs[e].y]
    const ushort2* pairs;  // over e in [rowptr[k], rowptr[k + 1])
};

struct Warp {
    DaTab t;
    int lane;
    const unsigned char* ex;  // [nc][3] exponents (shared memory)
    __device__ int deg(int k) const { return ex[3 * k] + ex[3 * k + 1] + ex[3 * k + 2]; }

    __device__ void set(double* a, double c0) const {
        for (int k = lane; k < t.nc; k += 32) a[k] = k == 0 ? c0 : 0.0;
        __syncwarp();
    }
    __device__ void copy(const double* a, double* b) const {
        for (int k = lane; k < t.nc; k += 32) b[k] = a[k];
        __syncwarp();
    }
    // b += s a
    __device__ void axpy(double s, const double* a, double* b) const {
        for (int k = lane; k < t.nc; k += 32) b[k] = fma(s, a[k], b[k]);
        __syncwarp();
    }
    // out = a b truncated at order p (out aliases neither)
    __device__ void mul(const double* a, const double* b, double* out) const {
        for (int k = lane; k < t.nc; k += 32) {
            double s = 0.0;
            for (int e = t.rowptr[k]; e < t.rowptr[k + 1]; ++e) {
                const ushort2 pr = t.pairs[e];
                s = fma(a[pr.x], b[pr.y], s);
            }
            out[k] = s;
        }
        __syncwarp();
    }
    // out = (a0 + abar)^e for abar without constant term: a0^e sum_k C(e, k) u^k with
    // u = abar / a0, by Horner's rule (u^k vanishes beyond order p); u and w are scratch
    __device__ void pow(double a0, const double* abar, double e, double* out, double* u, double* w) const {
        const double ia0 = 1.0 / a0;
        for (int k = lane; k < t.nc; k += 32) u[k] = k == 0 ? 0.0 : abar[k] * ia0;
        double cb[11];
        cb[0] = 1.0;
        for (int k = 1; k <= t.p; ++k) cb[k] = cb[k - 1] * (e - (k - 1)) / k;
        set(out, cb[t.p]);
        for (int k = t.p - 1; k >= 0; --k) {
            mul(u, out, w);
            for (int j = lane; j < t.nc; j += 32) out[j] = j == 0 ? w[j] + cb[k] : w[j];
            __syncwarp();
        }
        const double f = ::pow(a0, e);
        for (int k = lane; k < t.nc; k += 32) out[k] *= f;
        __syncwarp();
    }
    // out = phi o (g0, g1, g2) truncated at order p: sum over alpha of phi_alpha g0^a g1^b g2^c,
    // the monomials built by running products; X, XY, Z0, Z1 are scratch
    __device__ void compose(const double* phi, double* const* g, double* out, double* X, double* XY, double* Z0,
                            double* Z1) const {
        set(out, 0.0);
        set(X, 1.0);
        for (int a = 0; a <= t.p; ++a) {
            if (a > 0) {
                mul(X, g[0], Z0);
                copy(Z0, X);
            }
            copy(X, XY);
            for (int b = 0; b <= t.p - a; ++b) {
                if (b > 0) {
                    mul(XY, g[1], Z0);
                    copy(Z0, XY);
                }
                double* Zc = Z0;
                double* Zn = Z1;
                copy(XY, Zc);
                for (int c = 0; c <= t.p - a - b; ++c) {
                    if (c > 0) {
                        mul(Zc, g[2], Zn);
                        double* tmp = Zc;
                        Zc = Zn;
                        Zn = tmp;
                    }
                    axpy(phi[da_index(a, b, c)], Zc, out);
                }
            }
        }
    }
    // value and gradient of the polynomial phi at (x, y, z) (DA evaluation), on lane 0
    __device__ void eval(const double* phi, double x, double y, double z, double* out4) const {
        double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int k = lane; k < t.nc; k += 32) {
            const int a = ex[3 * k], b = ex[3 * k + 1], c = ex[3 * k + 2];
            double pa = 1.0, pb = 1.0, pc = 1.0, qa = 0.0, qb = 0.0, qc = 0.0;  // x^a and a x^(a-1), ...
            for (int i = 0; i < a; ++i) { qa = qa * x + pa; pa *= x; }
            for (int i = 0; i < b; ++i) { qb = qb * y + pb; pb *= y; }
            for (int i = 0; i < c; ++i) { qc = qc * z + pc; pc *= z; }
            const double f = phi[k];
            v = fma(f, pa * pb * pc, v);
            gx = fma(f, qa * pb * pc, gx);
            gy = fma(f, pa * qb * pc, gy);
            gz = fma(f, pa * pb * qc, gz);
        }
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_down_sync(0xffffffffu, v, o);
            gx += __shfl_down_sync(0xffffffffu, gx, o);
            gy += __shfl_down_sync(0xffffffffu, gy, o);
            gz += __shfl_down_sync(0xffffffffu, gz, o);
        }
        if (lane == 0) {
            out4[0] = v;
            out4[1] = gx;
            out4[2] = gy;
            out4[3] = gz;
        }
    }
    // the variable d_v as a DA vector, plus c0
    __device__ void var(double* a, int v, double c0) const {
        for (int k = lane; k < t.nc; k += 32) {
            const bool lin = deg(k) == 1 && ex[3 * k + v] == 1;
            a[k] = k == 0 ? c0 : (lin ? 1.0 : 0.0);
        }
        __syncwarp();
    }
    // |d|^2 = d0^2 + d1^2 + d2^2
    __device__ void square_norm(double* a) const {
        for (int k = lane; k < t.nc; k += 32) {
            const bool sq = deg(k) == 2 && (ex[3 * k] == 2 || ex[3 * k + 1] == 2 || ex[3 * k + 2] == 2);
            a[k] = sq ? 1.0 : 0.0;
        }
        __syncwarp();
    }
    // out_alpha *= s^|alpha|
    __device__ void scale_orders(double* a, double s) const {
        for (int k = lane; k < t.nc; k += 32) a[k] *= ::pow(s, (double)deg(k));
        __syncwarp();
    }
};


// first-order DA in the target offset (value and gradient), for M2P
struct D1 {
    double v, g[3];
};
__device__ D1 d1_mul(const D1& a, const D1& b) {
    D1 r;
    r.v = a.v * b.v;
    for (int i = 0; i < 3; ++i) r.g[i] = a.v * b.g[i] + a.g[i] * b.v;
    return r;
}

__global__ void __launch_bounds__(128) k_da_op(DaTab tab, int op, int64_t n, const double* __restrict__ A,
                                               const double* __restrict__ Bv, const int* __restrict__ oct,
                                               double* __restrict__ out) {
    extern __shared__ __align__(16) double da_smem[];
    const int nc = tab.nc;
    const int wpb = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ex = reinterpret_cast<unsigned char*>(da_smem + (size_t)wpb * kDaVecs * nc);
    for (int n_ = 0, k = 0; n_ <= tab.p; ++n_)
        for (int a = n_; a >= 0; --a)
            for (int b = n_ - a; b >= 0; --b, ++k)
                if (k % blockDim.x == threadIdx.x) {
                    ex[3 * k] = (unsigned char)a;
                    ex[3 * k + 1] = (unsigned char)b;
                    ex[3 * k + 2] = (unsigned char)(n_ - a - b);
                }
    __syncthreads();
    Warp W{tab, lane, ex};
    double* v[kDaVecs];
    for (int j = 0; j < kDaVecs; ++j) v[j] = da_smem + ((size_t)w * kDaVecs + j) * nc;
    for (int64_t i = (int64_t)blockIdx.x * wpb + w; i < n; i += (int64_t)gridDim.x * wpb) {
        switch (op) {
            case kDaP2M: {  // A: s (3), Bv: q
                const double s0 = A[3 * i], s1 = A[3 * i + 1], s2 = A[3 * i + 2];
                const double s2n = s0 * s0 + s1 * s1 + s2 * s2;
                W.square_norm(v[0]);
                for (int k = lane; k < nc; k += 32) {
                    double c = v[0][k] * s2n;
                    if (W.deg(k) == 1) c = -2.0 * (ex[3 * k] ? s0 : (ex[3 * k + 1] ? s1 : s2));
                    v[0][k] = c;
                }
                __syncwarp();
                W.pow(1.0, v[0], -0.5, v[1], v[2], v[3]);
                const double q = Bv[i];
                for (int k = lane; k < nc; k += 32) out[(size_t)i * nc + k] = q * v[1][k];
                break;
            }
            case kDaP2L: {  // A: w (3), Bv: q
                const double w0 = A[3 * i], w1 = A[3 * i + 1], w2 = A[3 * i + 2];
                W.square_norm(v[0]);
                for (int k = lane; k < nc; k += 32)
                    if (W.deg(k) == 1) v[0][k] = 2.0 * (ex[3 * k] ? w0 : (ex[3 * k + 1] ? w1 : w2));
                __syncwarp();
                W.pow(w0 * w0 + w1 * w1 + w2 * w2, v[0], -0.5, v[1], v[2], v[3]);
                const double q = Bv[i];
                for (int k = lane; k < nc; k += 32) out[(size_t)i * nc + k] = q * v[1][k];
                break;
            }
            case kDaL2P: {  // A: L (nc), Bv: x (3)
                W.eval(A + (size_t)i * nc, Bv[3 * i], Bv[3 * i + 1], Bv[3 * i + 2], out + 4 * (size_t)i);
                break;
            }
            case kDaM2P: {  // A: M (nc), Bv: s (3); first-order DA in the offset of s
                D1 s[3];
                for (int d = 0; d < 3; ++d) {
                    s[d].v = Bv[3 * i + d];
                    s[d].g[0] = s[d].g[1] = s[d].g[2] = 0.0;
                    s[d].g[d] = 1.0;
                }
                D1 r2 = d1_mul(s[0], s[0]);
                const D1 y2 = d1_mul(s[1], s[1]), z2 = d1_mul(s[2], s[2]);
                r2.v += y2.v + z2.v;
                for (int j = 0; j < 3; ++j) r2.g[j] += y2.g[j] + z2.g[j];
                D1 R, sR;  // 1/r2 and its square root
                R.v = 1.0 / r2.v;
                sR.v = sqrt(R.v);
                for (int j = 0; j < 3; ++j) {
                    R.g[j] = -R.v * R.v * r2.g[j];
                    sR.g[j] = 0.5 * R.g[j] / sR.v;
                }
                D1 d[3];
                for (int j = 0; j < 3; ++j) d[j] = d1_mul(s[j], R);
                // M(d) in first-order DA: value and d-gradient by DA evaluation, then the chain rule
                W.eval(A + (size_t)i * nc, d[0].v, d[1].v, d[2].v, v[0]);
                __syncwarp();
                if (lane == 0) {
                    D1 Md;
                    Md.v = v[0][0];
                    for (int j = 0; j < 3; ++j)
                        Md.g[j] = v[0][1] * d[0].g[j] + v[0][2] * d[1].g[j] + v[0][3] * d[2].g[j];
                    const D1 f = d1_mul(sR, Md);
                    double* o = out + 4 * (size_t)i;
                    o[0] = f.v;
                    o[1] = f.g[0];
                    o[2] = f.g[1];
                    o[3] = f.g[2];
                }
                __syncwarp();
                break;
            }
            case kDaM2M: {  // A: M (nc), oct
                const int o = oct[i];
                const double r0[3] = {0.5 - (o & 1), 0.5 - ((o >> 1) & 1), 0.5 - ((o >> 2) & 1)};
                const double r02 = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2];
                W.square_norm(v[0]);  // d'^2
                for (int k = lane; k < nc; k += 32) {
                    double c = r02 * v[0][k];
                    if (W.deg(k) == 1) c = 2.0 * (ex[3 * k] ? r0[0] : (ex[3 * k + 1] ? r0[1] : r0[2]));
                    v[1][k] = c;  // abar of 1/R
                }
                __syncwarp();
                W.pow(1.0, v[1], -1.0, v[2], v[14], v[15]);  // R
                W.pow(1.0, v[1], -0.5, v[3], v[14], v[15]);  // sqrt(R)
                for (int d = 0; d < 3; ++d) {                 // M1_d = (d'_d + d'^2 r0_d) R
                    W.var(v[13], d, 0.0);
                    W.axpy(r0[d], v[0], v[13]);
                    W.mul(v[13], v[2], v[4 + d]);
                }
                W.copy(A + (size_t)i * nc, v[7]);
                double* g[3] = {v[4], v[5], v[6]};
                W.compose(v[7], g, v[8], v[9], v[10], v[11], v[12]);
                W.mul(v[3], v[8], v[13]);
                W.scale_orders(v[13], 0.5);
                for (int k = lane; k < nc; k += 32) out[(size_t)i * nc + k] = v[13][k];
                break;
            }
            case kDaL2L: {  // A: L (nc), oct
                const int o = oct[i];
                for (int d = 0; d < 3; ++d) W.var(v[4 + d], d, 0.5 * (((o >> d) & 1) - 0.5));
                W.copy(A + (size_t)i * nc, v[7]);
                double* g[3] = {v[4], v[5], v[6]};
                W.compose(v[7], g, v[8], v[9], v[10], v[11], v[12]);
                W.scale_orders(v[8], 0.5);
                for (int k = lane; k < nc; k += 32) out[(size_t)i * nc + k] = v[8][k];
                break;
            }
            case kDaM2L: {  // A: M (nc), Bv: r0 (3)
                const double r0[3] = {Bv[3 * i], Bv[3 * i + 1], Bv[3 * i + 2]};
                const double r02 = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2];
                W.square_norm(v[0]);  // |r0 + d'|^2 = r0^2 + 2 r0.d' + d'^2
                for (int k = lane; k < nc; k += 32)
                    if (W.deg(k) == 1) v[0][k] = 2.0 * (ex[3 * k] ? r0[0] : (ex[3 * k + 1] ? r0[1] : r0[2]));
                __syncwarp();
                W.pow(r02, v[0], -1.0, v[2], v[14], v[15]);  // R
                W.pow(r02, v[0], -0.5, v[3], v[14], v[15]);  // sqrt(R)
                for (int d = 0; d < 3; ++d) {                // M2_d = (r0_d + d'_d) R
                    W.var(v[13], d, r0[d]);
                    W.mul(v[13], v[2], v[4 + d]);
                }
                W.copy(A + (size_t)i * nc, v[7]);
                double* g[3] = {v[4], v[5], v[6]};
                W.compose(v[7], g, v[8], v[9], v[10], v[11], v[12]);
                W.mul(v[3], v[8], v[13]);
                for (int k = lane; k < nc; k += 32) out[(size_t)i * nc + k] = v[13][k];
                break;
            }
        }
        __syncwarp();
    }
}

}  // namespace

// shared memory of one block of `warps` warps at `nc` coefficients
static size_t da_smem_bytes(int warps, int nc) {
    return (size_t)warps * kDaVecs * nc * sizeof(double) + (size_t)3 * nc + 16;
}

cudaError_t launch_da_op(const OrderData& od, int op, int64_t n, const double* a, const double* b, const int* oct,
                         double* out, int num_sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    DaTab tab{od.p, od.nc, od.mul_rowptr, od.mul_pairs};
    int warps = 4;
    while (warps > 1 && da_smem_bytes(warps, od.nc) > 200 * 1024) warps >>= 1;
    const size_t smem = da_smem_bytes(warps, od.nc);
    cudaError_t e = cudaFuncSetAttribute(k_da_op, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks_needed = (n + warps - 1) / warps;
    const int64_t cap = (int64_t)num_sms * 8;
    const unsigned grid = (unsigned)(blocks_needed < cap ? blocks_needed : cap);
    k_da_op<<<grid, 32 * warps, smem, s>>>(tab, op, n, a, b, oct, out);
    return cudaGetLastError();
}

}  // namespace dafmm
