// api.cu -- host runtime behind the C ABI of include/dafmm.h: contexts with an HBM budget,
// octree construction, the FMM evaluation sequence (Sec. 1) and the single-operator batches.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "check.cuh"
#include "da_common.cuh"
#include "internal.h"
#include "rot_lists.h"
#include "tc_ops.h"
#include "tree_common.cuh"

using namespace dafmm;

#include "api_types.h"

namespace {

const char* code_name(int c) {
    switch (c) {
        case DAFMM_ERR_INVALID_ARG: return "invalid argument";
        case DAFMM_ERR_UNSUPPORTED_ORDER: return "unsupported order";
        case DAFMM_ERR_OVER_BUDGET: return "over HBM budget";
        case DAFMM_ERR_CUDA: return "CUDA error";
        case DAFMM_ERR_TIMEOUT: return "timeout";
        case DAFMM_ERR_UNSUPPORTED: return "unsupported option";
        case DAFMM_ERR_NO_DEVICE: return "no CUDA device";
        case DAFMM_ERR_CHECK: return "index check failed";
    }
    return "error";
}

int fail(dafmm_ctx* c, int code, const std::string& msg) {
    if (c) c->err = std::string(code_name(code)) + ": " + msg;
    return code;
}

int cuda_fail(dafmm_ctx* c, cudaError_t e, const char* where) {
    return fail(c, DAFMM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, call, where)                                     \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

// every device allocation of a context goes through here (budget accounting)
int dev_alloc(dafmm_ctx* c, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return DAFMM_OK;
    bytes = (bytes + 255) / 256 * 256;
    if (c->arena_base) {
        size_t off = 0;
        if (!c->arena.alloc(bytes, &off))
            return fail(c, DAFMM_ERR_OVER_BUDGET, std::string(what) + " needs " + std::to_string(bytes) +
                                                      " bytes, largest free block of the pool " +
                                                      std::to_string(c->arena.largest_free()));
        *p = c->arena_base + off;
        c->in_use += bytes;
        return DAFMM_OK;
    }
    if (c->budget && c->in_use + bytes > c->budget)
        return fail(c, DAFMM_ERR_OVER_BUDGET, std::string(what) + " needs " + std::to_string(bytes) +
                                                  " bytes, budget left " + std::to_string(c->budget - c->in_use));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DAFMM_ERR_OVER_BUDGET, std::string(what) + ": cudaMalloc: " + cudaGetErrorString(e));
    }
    c->in_use += bytes;
    return DAFMM_OK;
}

void dev_free(dafmm_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    char* cp = static_cast<char*>(p);
    if (c->arena_base && cp >= c->arena_base && cp < c->arena_base + c->arena.size()) {
        bytes = c->arena.release((size_t)(cp - c->arena_base));
    } else {
        cudaFree(p);
        bytes = (bytes + 255) / 256 * 256;
    }
    c->in_use = c->in_use >= bytes ? c->in_use - bytes : 0;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t level_boxes(int l) { return (size_t)1 << (3 * l); }

// a device view of caller memory: either the pointer itself or a staged copy
struct Staged {
    dafmm_ctx* c = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool owned = false;
    ~Staged() {
        if (owned) dev_free(c, dev, bytes);
    }
};

int stage_in(dafmm_ctx* c, const void* src, size_t bytes, cudaStream_t s, Staged& out) {
    out.c = c;
    out.bytes = bytes;
    if (bytes == 0) return DAFMM_OK;
    if (is_device_ptr(src)) {
        out.dev = const_cast<void*>(src);
        return DAFMM_OK;
    }
    int rc = dev_alloc(c, &out.dev, bytes, "input staging");
    if (rc) return rc;
    out.owned = true;
    CK(c, cudaMemcpyAsync(out.dev, src, bytes, cudaMemcpyHostToDevice, s), "stage input");
    return DAFMM_OK;
}

// ---- per-order tables -----------------------------------------------------------------------
template <class T>
int upload(dafmm_ctx* c, T** dst, const T* src, size_t count, const char* what) {
    int rc = dev_alloc(c, (void**)dst, count * sizeof(T), what);
    if (rc) return rc;
    if (count) CK(c, cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice), what);
    return DAFMM_OK;
}

// M2L matrices by the octahedral symmetry of 1/|w|: for a signed axis permutation g,
// (g w)_d = sigma_d w_{pi(d)}, K_{g c}[b][a] = s(a) s(b) K_c[gamma(b)][gamma(a)] with
// gamma(e)_{pi(d)} = e_d and s(e) = prod_d sigma_d^{e_d}.  The 316 displacements fall into 16
// classes c = (|v| sorted descending); only those are generated by numerical DA.
__global__ void k_ksym(const short* __restrict__ keyc, const unsigned char* __restrict__ keyperm,
                       const unsigned char* __restrict__ keyneg, const short* __restrict__ gperm,
                       const unsigned char* __restrict__ par, double* __restrict__ K64, float* __restrict__ K32,
                       int nc, int ncp) {
    const int v = blockIdx.x;
    const int cls = keyc[v];
    if (cls < 0) return;  // a generated representative, or an adjacent (unused) displacement
    const short* g = gperm + (size_t)keyperm[v] * nc;
    const unsigned neg = keyneg[v];
    const double* Kc = K64 + (size_t)cls * nc * ncp;
    double* Kv = K64 + (size_t)v * nc * ncp;
    float* Kv32 = K32 + (size_t)v * nc * ncp;
    for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) {
        const int b = i / nc, a = i - b * nc;
        double x = Kc[(size_t)g[b] * ncp + g[a]];
        if (__popc((par[a] ^ par[b]) & neg) & 1) x = -x;
        Kv[(size_t)b * ncp + a] = x;
        Kv32[(size_t)b * ncp + a] = (float)x;
    }
}

int kgen_octahedral(dafmm_ctx* c, OrderData& od, int p, const OrderOps* ops, cudaStream_t s) {
    const int nc = od.nc;
    // exponents of each coefficient and their parity bits
    std::vector<int> ex(3 * nc);
    for (int n = 0; n <= p; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                const int k = da_index(a, b, n - a - b);
                ex[3 * k] = a; ex[3 * k + 1] = b; ex[3 * k + 2] = n - a - b;
            }
    std::vector<unsigned char> par(nc);
    for (int k = 0; k < nc; ++k) par[k] = (unsigned char)((ex[3 * k] & 1) | ((ex[3 * k + 1] & 1) << 1) | ((ex[3 * k + 2] & 1) << 2));
    // the 6 axis permutations pi (pi[d] = position of axis d in the class representative)
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    std::vector<short> gperm(6 * (size_t)nc);
    for (int q = 0; q < 6; ++q)
        for (int k = 0; k < nc; ++k) {
            int ge[3];
            for (int d = 0; d < 3; ++d) ge[perms[q][d]] = ex[3 * k + d];
            gperm[(size_t)q * nc + k] = (short)da_index(ge[0], ge[1], ge[2]);
        }
    std::vector<short> keyc(kNumKeys, -1), reps;
    std::vector<unsigned char> keyperm(kNumKeys, 0), keyneg(kNumKeys, 0);
    for (int key = 0; key < kNumKeys; ++key) {
        const int v[3] = {key / 49 - 3, (key / 7) % 7 - 3, key % 7 - 3};
        const int av[3] = {abs(v[0]), abs(v[1]), abs(v[2])};
        if (std::max(av[0], std::max(av[1], av[2])) <= 1) continue;
        int order[3] = {0, 1, 2};  // axes by |v| descending, ties by axis
        std::sort(order, order + 3, [&](int x, int y) { return av[x] != av[y] ? av[x] > av[y] : x < y; });
        int pi[3];
        for (int j = 0; j < 3; ++j) pi[order[j]] = j;
        const int ckey = (av[order[0]] + 3) * 49 + (av[order[1]] + 3) * 7 + (av[order[2]] + 3);
        int q = 0;
        while (!(perms[q][0] == pi[0] && perms[q][1] == pi[1] && perms[q][2] == pi[2])) ++q;
        unsigned neg = 0;
        for (int d = 0; d < 3; ++d)
            if (v[d] < 0) neg |= 1u << d;
        if (key == ckey) {
            reps.push_back((short)key);
        } else {
            keyc[key] = (short)ckey;
            keyperm[key] = (unsigned char)q;
            keyneg[key] = (unsigned char)neg;
        }
    }
    // device copies of the small tables (freed before returning)
    const size_t b_reps = reps.size() * sizeof(short), b_keyc = keyc.size() * sizeof(short), b_kb = kNumKeys,
                 b_g = gperm.size() * sizeof(short), b_par = (size_t)nc;
    char* tab = nullptr;
    const size_t total = 256 * 6 + b_reps + b_keyc + 2 * b_kb + b_g + b_par;
    int rc = dev_alloc(c, (void**)&tab, total, "symmetry tables");
    if (rc) return rc;
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes) {
        char* dst = tab + off;
        off += (bytes + 255) / 256 * 256;
        cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
        return dst;
    };
    const short* d_reps = (const short*)put(reps.data(), b_reps);
    const short* d_keyc = (const short*)put(keyc.data(), b_keyc);
    const unsigned char* d_kp = (const unsigned char*)put(keyperm.data(), b_kb);
    const unsigned char* d_kn = (const unsigned char*)put(keyneg.data(), b_kb);
    const short* d_g = (const short*)put(gperm.data(), b_g);
    const unsigned char* d_par = (const unsigned char*)put(par.data(), b_par);
    cudaError_t e = ops->kgen(od, d_reps, (int)reps.size(), s);
    if (e == cudaSuccess) {
        k_ksym<<<kNumKeys, 256, 0, s>>>(d_keyc, d_kp, d_kn, d_g, d_par, od.K64, od.K32, nc, od.ncp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(c, tab, total);
    if (e != cudaSuccess) return cuda_fail(c, e, "K generation");
    return DAFMM_OK;
}

int ensure_order(dafmm_ctx* c, int p, cudaStream_t s, bool need_k) {
    if (p < 0 || p > kMaxOrder) return fail(c, DAFMM_ERR_UNSUPPORTED_ORDER, "order " + std::to_string(p));
    OrderData& od = c->ord[p];
    const OrderOps* ops = order_ops(p);
    if (od.p < 0) {
        od.p = p;
        od.nc = ops->nc;
        od.ncp = ops->ncp;
        int rc;
        const HostShiftTable* tabs[2] = {&ops->m2m, &ops->l2l};
        for (int w = 0; w < 2; ++w) {
            const HostShiftTable& t = *tabs[w];
            std::vector<float> vf(t.val, t.val + t.nnz);
            int** rp = w == 0 ? &od.m2m_rowptr : &od.l2l_rowptr;
            unsigned short** col = w == 0 ? &od.m2m_col : &od.l2l_col;
            unsigned char** par = w == 0 ? &od.m2m_par : &od.l2l_par;
            double** val = w == 0 ? &od.m2m_val : &od.l2l_val;
            float** valf = w == 0 ? &od.m2m_valf : &od.l2l_valf;
            if ((rc = upload(c, rp, t.rowptr, (size_t)od.nc + 1, "shift table"))) return rc;
            if ((rc = upload(c, col, t.col, (size_t)t.nnz, "shift table"))) return rc;
            if ((rc = upload(c, par, t.par, (size_t)t.nnz, "shift table"))) return rc;
            if ((rc = upload(c, val, t.val, (size_t)t.nnz, "shift table"))) return rc;
            if ((rc = upload(c, valf, vf.data(), (size_t)t.nnz, "shift table"))) return rc;
            std::vector<int> rp8(8 * (size_t)od.nc + 1);
            shift_rp8(t, od.nc, rp8.data());
            if ((rc = upload(c, w == 0 ? &od.m2m_rp8 : &od.l2l_rp8, rp8.data(), rp8.size(), "shift table"))) return rc;
        }
        {  // the M2M of harmonic multipoles
            const HostShiftTable& t = ops->m2mh;
            std::vector<float> vf(t.val, t.val + t.nnz);
            if ((rc = upload(c, &od.m2mh_rowptr, t.rowptr, (size_t)od.nc + 1, "shift table"))) return rc;
            if ((rc = upload(c, &od.m2mh_col, t.col, (size_t)t.nnz, "shift table"))) return rc;
            if ((rc = upload(c, &od.m2mh_par, t.par, (size_t)t.nnz, "shift table"))) return rc;
            if ((rc = upload(c, &od.m2mh_val, t.val, (size_t)t.nnz, "shift table"))) return rc;
            if ((rc = upload(c, &od.m2mh_valf, vf.data(), (size_t)t.nnz, "shift table"))) return rc;
        }
        // DA product table: for each output k, the pairs (i, j) with e_i + e_j = e_k
        std::vector<int> ex(3 * od.nc);
        for (int n = 0; n <= p; ++n)
            for (int a = n; a >= 0; --a)
                for (int b = n - a; b >= 0; --b) {
                    int cc = n - a - b, k = da_index(a, b, cc);
                    ex[3 * k] = a; ex[3 * k + 1] = b; ex[3 * k + 2] = cc;
                }
        std::vector<int> rowptr(od.nc + 1, 0);
        std::vector<ushort2> pairs;
        for (int k = 0; k < od.nc; ++k) {
            rowptr[k] = (int)pairs.size();
            for (int i = 0; i < od.nc; ++i) {
                int r0 = ex[3 * k] - ex[3 * i], r1 = ex[3 * k + 1] - ex[3 * i + 1], r2 = ex[3 * k + 2] - ex[3 * i + 2];
                if (r0 < 0 || r1 < 0 || r2 < 0) continue;
                ushort2 pr;
                pr.x = (unsigned short)i;
                pr.y = (unsigned short)da_index(r0, r1, r2);
                pairs.push_back(pr);
            }
        }
        rowptr[od.nc] = (int)pairs.size();
        std::vector<short> minus(3 * od.nc);
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < od.nc; ++k) {
                int e[3] = {ex[3 * k], ex[3 * k + 1], ex[3 * k + 2]};
                if (e[d] == 0) {
                    minus[d * od.nc + k] = -1;
                } else {
                    e[d] -= 1;
                    minus[d * od.nc + k] = (short)da_index(e[0], e[1], e[2]);
                }
            }
        if ((rc = upload(c, &od.mul_rowptr, rowptr.data(), rowptr.size(), "product table"))) return rc;
        if ((rc = upload(c, &od.mul_pairs, pairs.data(), pairs.size(), "product table"))) return rc;
        od.mul_npairs = pairs.size();
        if ((rc = upload(c, &od.mul_minus, minus.data(), minus.size(), "product table"))) return rc;
    }
    if (need_k && !od.k_ready) {
        const size_t cnt = (size_t)kNumKeys * od.nc * od.ncp;
        int rc;
        if ((rc = dev_alloc(c, (void**)&od.K64, cnt * sizeof(double), "M2L matrices (FP64)"))) return rc;
        if ((rc = dev_alloc(c, (void**)&od.K32, cnt * sizeof(float), "M2L matrices (FP32)"))) return rc;
        CK(c, cudaMemsetAsync(od.K64, 0, cnt * sizeof(double), s), "K memset");
        CK(c, cudaMemsetAsync(od.K32, 0, cnt * sizeof(float), s), "K memset");
        if ((rc = kgen_octahedral(c, od, p, ops, s))) return rc;
        if (p >= 2) {
            const size_t cs = (size_t)kNumKeys * tc_npt(p) * od.ncp;
            if ((rc = dev_alloc(c, (void**)&od.Khi, cs * sizeof(float), "M2L matrices (TF32 split)"))) return rc;
            if ((rc = dev_alloc(c, (void**)&od.Klo, cs * sizeof(float), "M2L matrices (TF32 split)"))) return rc;
            CK(c, tc_split_rows(od.K64, kNumKeys, p, od.Khi, od.Klo, s), "K split");
            // dense M2M and L2L matrices of the 8 child octants (signs of Sec. 3.3 applied)
            const size_t ds = (size_t)8 * od.nc * od.ncp, ss = (size_t)8 * tc_npt(p) * od.ncp;
            std::vector<double> dense(ds);
            double* d64 = nullptr;
            if ((rc = dev_alloc(c, (void**)&d64, ds * sizeof(double), "shift tables"))) return rc;
            for (int w = 0; w < 2 && rc == 0; ++w) {
                const HostShiftTable& t = w == 0 ? ops->m2m : ops->l2l;
                std::fill(dense.begin(), dense.end(), 0.0);
                for (int oc = 0; oc < 8; ++oc)
                    for (int b = 0; b < od.nc; ++b)
                        for (int e = t.rowptr[b]; e < t.rowptr[b + 1]; ++e) {
                            const double v = (__builtin_popcount(t.par[e] & oc) & 1) ? -t.val[e] : t.val[e];
                            dense[((size_t)oc * od.nc + b) * od.ncp + t.col[e]] = v;
                        }
                float** hi = w == 0 ? &od.M2Mhi : &od.L2Lhi;
                float** lo = w == 0 ? &od.M2Mlo : &od.L2Llo;
                if ((rc = dev_alloc(c, (void**)hi, ss * sizeof(float), "shift tables (TF32 split)"))) break;
                if ((rc = dev_alloc(c, (void**)lo, ss * sizeof(float), "shift tables (TF32 split)"))) break;
                cudaError_t ce = cudaMemcpyAsync(d64, dense.data(), ds * sizeof(double), cudaMemcpyHostToDevice, s);
                if (ce == cudaSuccess) ce = tc_split_rows(d64, 8, p, *hi, *lo, s);
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);  // dense is reused for the next table
                if (ce != cudaSuccess) { rc = cuda_fail(c, ce, "shift tables"); break; }
            }
            dev_free(c, d64, ds * sizeof(double));
            if (rc) return rc;
        }
        // the tables are shared by every later evaluation, on any stream: finish them here
        CK(c, cudaStreamSynchronize(s), "K generation");
        od.k_ready = true;
    }
    return DAFMM_OK;
}

void free_order(dafmm_ctx* c, OrderData& od) {
    const int nc = od.nc;
    const OrderOps* ops = od.p >= 0 ? order_ops(od.p) : nullptr;
    if (!ops) return;
    for (int w = 0; w < 2; ++w) {
        const HostShiftTable& t = w == 0 ? ops->m2m : ops->l2l;
        dev_free(c, w == 0 ? (void*)od.m2m_rowptr : (void*)od.l2l_rowptr, (nc + 1) * sizeof(int));
        dev_free(c, w == 0 ? (void*)od.m2m_col : (void*)od.l2l_col, t.nnz * sizeof(unsigned short));
        dev_free(c, w == 0 ? (void*)od.m2m_par : (void*)od.l2l_par, t.nnz);
        dev_free(c, w == 0 ? (void*)od.m2m_val : (void*)od.l2l_val, t.nnz * sizeof(double));
        dev_free(c, w == 0 ? (void*)od.m2m_valf : (void*)od.l2l_valf, t.nnz * sizeof(float));
        dev_free(c, w == 0 ? (void*)od.m2m_rp8 : (void*)od.l2l_rp8, (8 * (size_t)nc + 1) * sizeof(int));
    }
    {
        const HostShiftTable& t = ops->m2mh;
        dev_free(c, od.m2mh_rowptr, od.m2mh_rowptr ? (nc + 1) * sizeof(int) : 0);
        dev_free(c, od.m2mh_col, od.m2mh_col ? t.nnz * sizeof(unsigned short) : 0);
        dev_free(c, od.m2mh_par, od.m2mh_par ? (size_t)t.nnz : 0);
        dev_free(c, od.m2mh_val, od.m2mh_val ? t.nnz * sizeof(double) : 0);
        dev_free(c, od.m2mh_valf, od.m2mh_valf ? t.nnz * sizeof(float) : 0);
    }
    dev_free(c, od.mul_rowptr, ((size_t)nc + 1) * sizeof(int));
    dev_free(c, od.mul_pairs, od.mul_npairs * sizeof(ushort2));
    dev_free(c, od.mul_minus, (size_t)3 * nc * sizeof(short));
    const size_t cnt = (size_t)kNumKeys * od.nc * od.ncp;
    dev_free(c, od.K64, od.K64 ? cnt * sizeof(double) : 0);
    dev_free(c, od.K32, od.K32 ? cnt * sizeof(float) : 0);
    if (od.Kh16) {
        const size_t c16 = (size_t)kNumKeys * tc_npt(od.p) * tc_rowlen16(od.p) * 2;
        dev_free(c, od.Kh16, c16);
        dev_free(c, od.Kl16, c16);
        dev_free(c, od.k16_inv_r, (size_t)tc_npt(od.p) * sizeof(float));
        dev_free(c, od.k16_inv_c, (size_t)kNumKeys * sizeof(float));
    }
    if (od.Kh16h) {
        const size_t c16 = (size_t)kNumKeys * tc_npt_h(od.p) * tc_rowlen16h(od.p) * 2;
        const size_t nstep = (size_t)(ncoef_of(od.p) - nharm_of(od.p));
        dev_free(c, od.Kh16h, c16);
        dev_free(c, od.Kl16h, c16);
        dev_free(c, od.k16h_inv_r, (size_t)tc_npt_h(od.p) * sizeof(float));
        dev_free(c, od.k16h_inv_c, (size_t)kNumKeys * sizeof(float));
        dev_free(c, od.hx_step, std::max<size_t>(nstep, 1) * sizeof(int4));
        dev_free(c, od.hx_w, std::max<size_t>(nstep, 1) * sizeof(float2));
        dev_free(c, od.hx_w64, std::max<size_t>(nstep, 1) * sizeof(double2));
        const size_t ctf = (size_t)kNumKeys * tc_npt_h(od.p) * harm_row(od.p) * sizeof(float);
        dev_free(c, od.Khih, ctf);
        dev_free(c, od.Kloh, ctf);
    }
    if (od.Khi) {
        const size_t cs = (size_t)kNumKeys * tc_npt(od.p) * od.ncp;
        dev_free(c, od.Khi, cs * sizeof(float));
        dev_free(c, od.Klo, cs * sizeof(float));
        const size_t ss = (size_t)8 * tc_npt(od.p) * od.ncp * sizeof(float);
        dev_free(c, od.M2Mhi, ss); dev_free(c, od.M2Mlo, ss);
        dev_free(c, od.L2Lhi, ss); dev_free(c, od.L2Llo, ss);
    }
    if (od.rot_T) {
        dev_free(c, od.rot_T, (size_t)kNumKeys * 4 * ops->rot_tsz * sizeof(double));
        dev_free(c, od.rot_rho, (size_t)kNumKeys * sizeof(int));
        dev_free(c, od.ax_rowptr, ((size_t)nc + 1) * sizeof(int));
        dev_free(c, od.ax_col, (size_t)od.ax_nnz * sizeof(unsigned short));
        dev_free(c, od.ax_val, (size_t)od.n_rho * od.ax_nnz * sizeof(double));
        dev_free(c, od.rot_lx, (size_t)od.rot_len[0] * 32 * sizeof(uint2));
        dev_free(c, od.rot_lz, (size_t)od.rot_len[1] * 32 * sizeof(uint2));
        dev_free(c, od.rot_la, (size_t)od.rot_len[2] * 32 * sizeof(uint2));
        dev_free(c, od.rot_lxh, (size_t)od.rot_lenh[0] * 32 * sizeof(uint2));
        dev_free(c, od.rot_lzh, (size_t)od.rot_lenh[1] * 32 * sizeof(uint2));
        dev_free(c, od.rot_lah, (size_t)od.rot_lenh[2] * 32 * sizeof(uint2));
        const size_t nhs = std::max<size_t>((size_t)(ncoef_of(od.p) - nharm_of(od.p)), 1);
        dev_free(c, od.hxr_step, nhs * sizeof(int4));
        dev_free(c, od.hxr_w, nhs * sizeof(double2));
        dev_free(c, od.rot_Tf, (size_t)kNumKeys * 4 * ops->rot_tsz * sizeof(float2));
        dev_free(c, od.ax_valf, (size_t)od.n_rho * od.ax_nnz * sizeof(float2));
    }
    od = OrderData();
}

// F16 splits of the M2L matrices of an order (made once, on first use)
int ensure_k16(dafmm_ctx* c, int p, cudaStream_t s) {
    OrderData& od = c->ord[p];
    if (od.Kh16) return DAFMM_OK;
    const int npt = tc_npt(p);
    const size_t c16 = (size_t)kNumKeys * npt * tc_rowlen16(p) * 2;
    int rc;
    void *hi = nullptr, *lo = nullptr;
    float *ir = nullptr, *ic = nullptr, *scratch = nullptr;
    if ((rc = dev_alloc(c, &hi, c16, "M2L matrices (F16 split)")) || (rc = dev_alloc(c, &lo, c16, "M2L matrices (F16 split)")) ||
        (rc = dev_alloc(c, (void**)&ir, (size_t)npt * sizeof(float), "M2L matrix factors")) ||
        (rc = dev_alloc(c, (void**)&ic, (size_t)kNumKeys * sizeof(float), "M2L matrix factors")) ||
        (rc = dev_alloc(c, (void**)&scratch, ((size_t)npt + kNumKeys) * sizeof(float), "M2L matrix factors"))) {
        dev_free(c, hi, c16); dev_free(c, lo, c16);
        dev_free(c, ir, (size_t)npt * sizeof(float)); dev_free(c, ic, (size_t)kNumKeys * sizeof(float));
        dev_free(c, scratch, ((size_t)npt + kNumKeys) * sizeof(float));
        return rc;
    }
    cudaError_t e = tc_prepare_k16(od.K64, kNumKeys, p, hi, lo, ir, ic, scratch, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // shared by every later evaluation, on any stream
    dev_free(c, scratch, ((size_t)npt + kNumKeys) * sizeof(float));
    if (e != cudaSuccess) {
        dev_free(c, hi, c16); dev_free(c, lo, c16);
        dev_free(c, ir, (size_t)npt * sizeof(float)); dev_free(c, ic, (size_t)kNumKeys * sizeof(float));
        return cuda_fail(c, e, "M2L matrices (F16 split)");
    }
    od.Kh16 = hi;
    od.Kl16 = lo;
    od.k16_inv_r = ir;
    od.k16_inv_c = ic;
    return DAFMM_OK;
}

// The steps that restore an expansion's coefficients of z exponent >= 2 from its free ones by
// Laplace's equation, in order of increasing z exponent: step (i, i1, i2, c) sets
// a[i] = w1 a[i1] + w2 a[i2] with w1 = -(a+2)(a+1) / (c(c-1)), w2 = -(b+2)(b+1) / (c(c-1)) for
// coefficient i = (a, b, c); those of z exponent c are [cst[c], cst[c + 1])
static void harm_steps(int p, std::vector<int4>& step, std::vector<double2>& w, int* cst) {
    const int nc = ncoef_of(p);
    std::vector<int> ea(nc), eb(nc), ec(nc);
    for (int n = 0; n <= p; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                const int cc = n - a - b, i = da_index(a, b, cc);
                ea[i] = a; eb[i] = b; ec[i] = cc;
            }
    step.clear();
    w.clear();
    for (int k = 0; k < kMaxOrder + 3; ++k) cst[k] = 0;
    for (int cz = 2; cz <= p + 1; ++cz) {
        cst[cz] = (int)step.size();
        for (int i = 0; i < nc; ++i) {
            if (ec[i] != cz) continue;
            const int a = ea[i], b = eb[i];
            const double d = (double)cz * (cz - 1);
            step.push_back(make_int4(i, da_index(a + 2, b, cz - 2), da_index(a, b + 2, cz - 2), cz));
            w.push_back(make_double2(-(double)(a + 2) * (a + 1) / d, -(double)(b + 2) * (b + 1) / d));
        }
    }
    cst[p + 2] = (int)step.size();
}

// The M2L in the harmonic basis (made once per order, on first use): the steps that restore the
// coefficients of z exponent >= 2 from the free ones (Laplace's equation, in order of increasing
// z exponent), the expansion matrix X [nc][nh] they define (FP64, for the matrices only), and
// the F16 and TF32 splits of the matrices restricted to the free output coefficients and
// composed with X
int ensure_k16h(dafmm_ctx* c, int p, cudaStream_t s) {
    OrderData& od = c->ord[p];
    if (od.Kh16h) return DAFMM_OK;
    const int nc = ncoef_of(p), nh = nharm_of(p), nhp = harm_row(p);
    const int npt = tc_npt_h(p), rowlen = tc_rowlen16h(p);
    std::vector<int4> step;
    std::vector<double2> w64;
    int cst[kMaxOrder + 3];
    harm_steps(p, step, w64, cst);
    std::vector<float2> w(w64.size());
    std::vector<double> X((size_t)nc * nh, 0.0);
    for (int k = 0; k < nh; ++k) X[(size_t)harm_full_index(k) * nh + k] = 1.0;
    for (size_t q = 0; q < step.size(); ++q) {
        const int i = step[q].x, i1 = step[q].y, i2 = step[q].z;
        w[q] = make_float2((float)w64[q].x, (float)w64[q].y);
        for (int k = 0; k < nh; ++k)
            X[(size_t)i * nh + k] = w64[q].x * X[(size_t)i1 * nh + k] + w64[q].y * X[(size_t)i2 * nh + k];
    }
    const size_t nstep = std::max<size_t>(step.size(), 1);
    const size_t c16 = (size_t)kNumKeys * npt * rowlen * 2;
    const size_t xb = (size_t)nc * nh * sizeof(double), khb = (size_t)kNumKeys * nh * nhp * sizeof(double);
    int rc;
    void *hi = nullptr, *lo = nullptr, *xd = nullptr, *khd = nullptr;
    float *ir = nullptr, *icv = nullptr, *scratch = nullptr, *thi = nullptr, *tlo = nullptr;
    const size_t ctf = (size_t)kNumKeys * npt * nhp * sizeof(float);
    int4* stp = nullptr;
    float2* wd = nullptr;
    double2* wd64 = nullptr;
    auto release = [&]() {
        dev_free(c, hi, hi ? c16 : 0); dev_free(c, lo, lo ? c16 : 0);
        dev_free(c, ir, ir ? (size_t)npt * sizeof(float) : 0);
        dev_free(c, icv, icv ? (size_t)kNumKeys * sizeof(float) : 0);
        dev_free(c, stp, stp ? nstep * sizeof(int4) : 0);
        dev_free(c, wd, wd ? nstep * sizeof(float2) : 0);
        dev_free(c, wd64, wd64 ? nstep * sizeof(double2) : 0);
        dev_free(c, thi, thi ? ctf : 0); dev_free(c, tlo, tlo ? ctf : 0);
    };
    auto release_scratch = [&]() {
        dev_free(c, xd, xd ? xb : 0);
        dev_free(c, khd, khd ? khb : 0);
        dev_free(c, scratch, scratch ? ((size_t)npt + kNumKeys) * sizeof(float) : 0);
    };
    if ((rc = dev_alloc(c, &hi, c16, "M2L matrices (harmonic, F16 split)")) ||
        (rc = dev_alloc(c, &lo, c16, "M2L matrices (harmonic, F16 split)")) ||
        (rc = dev_alloc(c, (void**)&ir, (size_t)npt * sizeof(float), "M2L matrix factors")) ||
        (rc = dev_alloc(c, (void**)&icv, (size_t)kNumKeys * sizeof(float), "M2L matrix factors")) ||
        (rc = dev_alloc(c, (void**)&stp, nstep * sizeof(int4), "harmonic expansion")) ||
        (rc = dev_alloc(c, (void**)&wd, nstep * sizeof(float2), "harmonic expansion")) ||
        (rc = dev_alloc(c, (void**)&wd64, nstep * sizeof(double2), "harmonic expansion")) ||
        (rc = dev_alloc(c, (void**)&thi, ctf, "M2L matrices (harmonic, TF32 split)")) ||
        (rc = dev_alloc(c, (void**)&tlo, ctf, "M2L matrices (harmonic, TF32 split)")) ||
        (rc = dev_alloc(c, &xd, xb, "harmonic expansion (scratch)")) ||
        (rc = dev_alloc(c, &khd, khb, "M2L matrices (harmonic, scratch)")) ||
        (rc = dev_alloc(c, (void**)&scratch, ((size_t)npt + kNumKeys) * sizeof(float), "M2L matrix factors"))) {
        release();
        release_scratch();
        return rc;
    }
    cudaError_t e = cudaMemcpyAsync(xd, X.data(), xb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !step.empty())
        e = cudaMemcpyAsync(stp, step.data(), step.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !w.empty())
        e = cudaMemcpyAsync(wd, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !w64.empty())
        e = cudaMemcpyAsync(wd64, w64.data(), w64.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = tc_prepare_k16h(od.K64, kNumKeys, p, static_cast<const double*>(xd), static_cast<double*>(khd), hi, lo, ir,
                            icv, scratch, thi, tlo, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors die with this call
    release_scratch();
    if (e != cudaSuccess) {
        release();
        return cuda_fail(c, e, "M2L matrices (harmonic)");
    }
    od.Kh16h = hi;
    od.Kl16h = lo;
    od.k16h_inv_r = ir;
    od.k16h_inv_c = icv;
    od.hx_step = stp;
    od.hx_w = wd;
    od.hx_w64 = wd64;
    od.Khih = thi;
    od.Kloh = tlo;
    for (int k = 0; k < kMaxOrder + 3; ++k) od.hx_cst[k] = cst[k];
    return DAFMM_OK;
}

// tables of the M2L by rotation (Sec. 3.4) of an order (made once, on first use): the four
// substitution tables of every displacement key, and the axial matrices of the distinct
// lengths |v| as their structural non-zeros (row b, column a: b_y >= a_y, b_z >= a_z, both
// differences even), the values taken from the K generation along the x axis
int ensure_rotation(dafmm_ctx* c, int p, cudaStream_t s) {
    OrderData& od = c->ord[p];
    if (od.rot_T) return DAFMM_OK;
    const OrderOps* ops = order_ops(p);
    const int nc = ncoef_of(p), ncp = ncp_of(p);
    // the axial matrices' structure and the kernel's task lists (rot_lists.h)
    const RotStructure rs = rot_structure(p);
    const std::vector<int>& rowptr = rs.rowptr;
    const std::vector<unsigned short>& col = rs.col;
    const int nnz = (int)col.size();
    std::vector<int> rho_of(kNumKeys, 0), len2;
    for (int key = 0; key < kNumKeys; ++key) {
        const int vx = key / 49 - 3, vy = (key / 7) % 7 - 3, vz = key % 7 - 3;
        if (std::max(std::abs(vx), std::max(std::abs(vy), std::abs(vz))) <= 1) continue;
        const int r2 = vx * vx + vy * vy + vz * vz;
        auto it = std::find(len2.begin(), len2.end(), r2);
        rho_of[key] = (int)(it - len2.begin());
        if (it == len2.end()) len2.push_back(r2);
    }
    const int nrho = (int)len2.size();
    static_assert(sizeof(RotTask) == sizeof(uint2), "task layout");
    const std::vector<RotTask>& lx = rs.lx;
    const std::vector<RotTask>& lz = rs.lz;
    const std::vector<RotTask>& la = rs.la;
    const int len_x = rs.len[0], len_z = rs.len[1], len_a = rs.len[2];
    // the harmonic form: lists of the free outputs, and the steps restoring the others
    const RotStructure rsh = rot_structure(p, true);
    std::vector<int4> hstep;
    std::vector<double2> hw;
    int hcst[kMaxOrder + 3];
    harm_steps(p, hstep, hw, hcst);
    const size_t nhstep = std::max<size_t>(hstep.size(), 1);
    std::vector<double> r0s(3 * (size_t)nrho, 0.0);
    for (int r = 0; r < nrho; ++r) r0s[3 * r] = std::sqrt((double)len2[r]);
    const size_t tbytes = (size_t)kNumKeys * 4 * ops->rot_tsz * sizeof(double);
    const size_t kbytes = (size_t)nrho * nc * ncp * sizeof(double);
    double *T = nullptr, *val = nullptr, *d_r0s = nullptr, *Ks = nullptr;
    int *rho = nullptr, *rp = nullptr;
    unsigned short* cl = nullptr;
    uint2 *dlx = nullptr, *dlz = nullptr, *dla = nullptr, *dlxh = nullptr, *dlzh = nullptr, *dlah = nullptr;
    int4* dhs = nullptr;
    double2* dhw = nullptr;
    int rc;
    auto release = [&]() {
        dev_free(c, dlx, lx.size() * sizeof(uint2));
        dev_free(c, dlz, lz.size() * sizeof(uint2));
        dev_free(c, dla, la.size() * sizeof(uint2));
        dev_free(c, dlxh, dlxh ? rsh.lx.size() * sizeof(uint2) : 0);
        dev_free(c, dlzh, dlzh ? rsh.lz.size() * sizeof(uint2) : 0);
        dev_free(c, dlah, dlah ? rsh.la.size() * sizeof(uint2) : 0);
        dev_free(c, dhs, dhs ? nhstep * sizeof(int4) : 0);
        dev_free(c, dhw, dhw ? nhstep * sizeof(double2) : 0);
        dev_free(c, T, tbytes);
        dev_free(c, val, (size_t)nrho * nnz * sizeof(double));
        dev_free(c, rho, (size_t)kNumKeys * sizeof(int));
        dev_free(c, rp, ((size_t)nc + 1) * sizeof(int));
        dev_free(c, cl, (size_t)nnz * sizeof(unsigned short));
    };
    if ((rc = dev_alloc(c, (void**)&T, tbytes, "rotation tables")) ||
        (rc = dev_alloc(c, (void**)&val, (size_t)nrho * nnz * sizeof(double), "axial M2L matrices")) ||
        (rc = dev_alloc(c, (void**)&rho, (size_t)kNumKeys * sizeof(int), "rotation tables")) ||
        (rc = dev_alloc(c, (void**)&rp, ((size_t)nc + 1) * sizeof(int), "axial M2L matrices")) ||
        (rc = dev_alloc(c, (void**)&cl, (size_t)nnz * sizeof(unsigned short), "axial M2L matrices")) ||
        (rc = dev_alloc(c, (void**)&dlx, lx.size() * sizeof(uint2), "rotation task lists")) ||
        (rc = dev_alloc(c, (void**)&dlz, lz.size() * sizeof(uint2), "rotation task lists")) ||
        (rc = dev_alloc(c, (void**)&dla, la.size() * sizeof(uint2), "rotation task lists")) ||
        (rc = dev_alloc(c, (void**)&dlxh, rsh.lx.size() * sizeof(uint2), "rotation task lists")) ||
        (rc = dev_alloc(c, (void**)&dlzh, rsh.lz.size() * sizeof(uint2), "rotation task lists")) ||
        (rc = dev_alloc(c, (void**)&dlah, rsh.la.size() * sizeof(uint2), "rotation task lists")) ||
        (rc = dev_alloc(c, (void**)&dhs, nhstep * sizeof(int4), "harmonic expansion")) ||
        (rc = dev_alloc(c, (void**)&dhw, nhstep * sizeof(double2), "harmonic expansion"))) {
        release();
        return rc;
    }
    if ((rc = dev_alloc(c, (void**)&d_r0s, r0s.size() * sizeof(double), "rotation scratch")) ||
        (rc = dev_alloc(c, (void**)&Ks, kbytes, "rotation scratch"))) {
        dev_free(c, d_r0s, r0s.size() * sizeof(double));
        release();
        return rc;
    }
    od.rot_T = T; od.rot_rho = rho; od.ax_rowptr = rp; od.ax_col = cl; od.ax_val = val;
    od.ax_nnz = nnz; od.n_rho = nrho;
    od.rot_lx = dlx; od.rot_lz = dlz; od.rot_la = dla;
    od.rot_len[0] = len_x; od.rot_len[1] = len_z; od.rot_len[2] = len_a;
    od.rot_lxh = dlxh; od.rot_lzh = dlzh; od.rot_lah = dlah;
    od.rot_lenh[0] = rsh.len[0]; od.rot_lenh[1] = rsh.len[1]; od.rot_lenh[2] = rsh.len[2];
    od.hxr_step = dhs; od.hxr_w = dhw;
    for (int k = 0; k < kMaxOrder + 3; ++k) od.hxr_cst[k] = hcst[k];
    cudaError_t e = cudaMemcpyAsync(rho, rho_of.data(), rho_of.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dlxh, rsh.lx.data(), rsh.lx.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dlzh, rsh.lz.data(), rsh.lz.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dlah, rsh.la.data(), rsh.la.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !hstep.empty())
        e = cudaMemcpyAsync(dhs, hstep.data(), hstep.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !hw.empty())
        e = cudaMemcpyAsync(dhw, hw.data(), hw.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rp, rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cl, col.data(), col.size() * sizeof(unsigned short), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_r0s, r0s.data(), r0s.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dlx, lx.data(), lx.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dlz, lz.data(), lz.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dla, la.data(), la.size() * sizeof(uint2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = ops->rot_setup(od, d_r0s, nrho, Ks, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // shared by every later evaluation, on any stream
    dev_free(c, d_r0s, r0s.size() * sizeof(double));
    dev_free(c, Ks, kbytes);
    if (e != cudaSuccess) {
        release();
        od.rot_T = nullptr; od.rot_rho = nullptr; od.ax_rowptr = nullptr; od.ax_col = nullptr; od.ax_val = nullptr;
        od.rot_lx = od.rot_lz = od.rot_la = nullptr;
        od.rot_lxh = od.rot_lzh = od.rot_lah = nullptr;
        od.hxr_step = nullptr;
        od.hxr_w = nullptr;
        return cuda_fail(c, e, "rotation tables");
    }
    return DAFMM_OK;
}

// float-float copies of the rotation tables and axial values (the DAFMM_FF mode's M2L)
int ensure_rotation_ff(dafmm_ctx* c, int p, cudaStream_t s) {
    int rc;
    if ((rc = ensure_rotation(c, p, s))) return rc;
    OrderData& od = c->ord[p];
    if (od.rot_Tf) return DAFMM_OK;
    const OrderOps* ops = order_ops(p);
    const size_t nt = (size_t)kNumKeys * 4 * ops->rot_tsz, na = (size_t)od.n_rho * od.ax_nnz;
    float2 *T = nullptr, *A = nullptr;
    if ((rc = dev_alloc(c, (void**)&T, nt * sizeof(float2), "rotation tables (float-float)"))) return rc;
    if ((rc = dev_alloc(c, (void**)&A, na * sizeof(float2), "axial M2L matrices (float-float)"))) {
        dev_free(c, T, nt * sizeof(float2));
        return rc;
    }
    cudaError_t e = ops->to_ff(od.rot_T, T, nt, s);
    if (e == cudaSuccess) e = ops->to_ff(od.ax_val, A, na, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // shared by every later evaluation, on any stream
    if (e != cudaSuccess) {
        dev_free(c, T, nt * sizeof(float2));
        dev_free(c, A, na * sizeof(float2));
        return cuda_fail(c, e, "rotation tables (float-float)");
    }
    od.rot_Tf = T;
    od.ax_valf = A;
    return DAFMM_OK;
}

// ---- expansions --------------------------------------------------------------------------------
void free_expansions(dafmm_tree* t) {
    dafmm_ctx* c = t->ctx;
    Expansions& e = t->ex;
    if (e.p < 0) return;
    const int ncp = ncp_of(e.p);
    for (int l = 0; l <= e.depth; ++l) {
        const size_t cnt = level_boxes(l) * ncp;
        dev_free(c, e.M[l], e.M[l] ? cnt * sizeof(double) : 0);
        dev_free(c, e.L[l], e.L[l] ? cnt * sizeof(double) : 0);
        dev_free(c, e.Mf[l], e.Mf[l] ? cnt * sizeof(float) : 0);
        dev_free(c, e.Mhi[l], e.Mhi[l] ? cnt * sizeof(float) : 0);
        dev_free(c, e.Mlo[l], e.Mlo[l] ? cnt * sizeof(float) : 0);
        dev_free(c, e.Lhi[l], e.Lhi[l] ? cnt * sizeof(float) : 0);
        dev_free(c, e.Llo[l], e.Llo[l] ? cnt * sizeof(float) : 0);
        const size_t c16 = level_boxes(l) * (size_t)tc_rowlen16(e.p) * 2;
        dev_free(c, e.Mh16[l], c16);
        dev_free(c, e.Ml16[l], c16);
        dev_free(c, e.Minv[l], level_boxes(l) * sizeof(float));
        dev_free(c, e.Lh[l], e.Lh[l] ? level_boxes(l) * harm_row(e.p) * sizeof(float) : 0);
    }
    e = Expansions();
}

int ensure_expansions(dafmm_tree* t, int p, cudaStream_t s) {
    if (t->ex.p == p) return DAFMM_OK;
    free_expansions(t);
    dafmm_ctx* c = t->ctx;
    const int ncp = ncp_of(p);
    t->ex.p = p;
    t->ex.depth = t->depth;
    for (int l = 2; l <= t->depth; ++l) {
        const size_t cnt = level_boxes(l) * ncp;
        int rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.M[l], cnt * sizeof(double), "multipoles"))) return rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.L[l], cnt * sizeof(double), "locals"))) return rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.Mf[l], cnt * sizeof(float), "multipoles (FP32)"))) return rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.Mhi[l], cnt * sizeof(float), "multipoles (TF32 split)"))) return rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.Mlo[l], cnt * sizeof(float), "multipoles (TF32 split)"))) return rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.Lhi[l], cnt * sizeof(float), "locals (TF32 split)"))) return rc;
        if ((rc = dev_alloc(c, (void**)&t->ex.Llo[l], cnt * sizeof(float), "locals (TF32 split)"))) return rc;
        CK(c, cudaMemsetAsync(t->ex.M[l], 0, cnt * sizeof(double), s), "memset");
        CK(c, cudaMemsetAsync(t->ex.L[l], 0, cnt * sizeof(double), s), "memset");
        CK(c, cudaMemsetAsync(t->ex.Mf[l], 0, cnt * sizeof(float), s), "memset");
        CK(c, cudaMemsetAsync(t->ex.Mhi[l], 0, cnt * sizeof(float), s), "memset");
        CK(c, cudaMemsetAsync(t->ex.Mlo[l], 0, cnt * sizeof(float), s), "memset");
        CK(c, cudaMemsetAsync(t->ex.Lhi[l], 0, cnt * sizeof(float), s), "memset");
        CK(c, cudaMemsetAsync(t->ex.Llo[l], 0, cnt * sizeof(float), s), "memset");
    }
    return DAFMM_OK;
}

// the F16 multipole splits of every level of a uniform tree (made on first use)
int ensure_f16_levels(dafmm_tree* t, cudaStream_t s) {
    (void)s;
    dafmm_ctx* c = t->ctx;
    Expansions& e = t->ex;
    for (int l = 2; l <= e.depth; ++l) {
        if (e.Mh16[l]) continue;
        const size_t c16 = level_boxes(l) * (size_t)tc_rowlen16(e.p) * 2;
        int rc;
        if ((rc = dev_alloc(c, &e.Mh16[l], c16, "multipoles (F16 split)"))) return rc;
        if ((rc = dev_alloc(c, &e.Ml16[l], c16, "multipoles (F16 split)"))) return rc;
        if ((rc = dev_alloc(c, (void**)&e.Minv[l], level_boxes(l) * sizeof(float), "multipole factors"))) return rc;
    }
    return DAFMM_OK;
}

// the harmonic-basis M2L's output rows per level (FP32, harm_row floats per box)
int ensure_lh_levels(dafmm_tree* t) {
    dafmm_ctx* c = t->ctx;
    Expansions& e = t->ex;
    for (int l = 2; l <= e.depth; ++l) {
        int rc;
        if (!e.Lh[l] &&
            (rc = dev_alloc(c, (void**)&e.Lh[l], level_boxes(l) * harm_row(e.p) * sizeof(float), "locals (harmonic)")))
            return rc;
    }
    return DAFMM_OK;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

size_t tree_bytes(int64_t n, int depth) {
    const size_t nl = level_boxes(depth);
    return (size_t)n * (4 * sizeof(double) + sizeof(int)) + 2 * xq_records(n, (int64_t)nl) * sizeof(float4) +
           (nl + 1) * sizeof(int);
}


// ---- adaptive trees -----------------------------------------------------------------------------
AdaptiveBuild abuild(dafmm_tree* t, const uint64_t* keys) {
    AdaptiveBuild ab;
    ab.keys = keys;
    ab.root = t->a_root;
    ab.level = t->a_level;
    ab.ijk = t->a_ijk;
    ab.parent = t->a_parent;
    ab.child = t->a_child;
    ab.pbeg = t->a_pbeg;
    ab.pend = t->a_pend;
    ab.colleague = t->a_colleague;
#if defined(DAFMM_CHECK)
    ab.cap = t->cap;
    ab.nbox = t->nbox;
#endif
    return ab;
}

AdaptiveView aview(const dafmm_tree* t) {
    AdaptiveView v;
    v.nbox = t->nbox;
    v.level = t->a_level;
    v.ijk = t->a_ijk;
    v.parent = t->a_parent;
    v.child = t->a_child;
    v.pbeg = t->a_pbeg;
    v.pend = t->a_pend;
    v.colleague = t->a_colleague;
    v.u_ptr = t->u_ptr; v.u_idx = t->u_idx;
    v.w_ptr = t->w_ptr; v.w_idx = t->w_idx;
    v.x_ptr = t->x_ptr; v.x_idx = t->x_idx;
    v.geom = t->a_geom;
    v.xq0 = t->a_xq0;
    v.x = t->x; v.y = t->y; v.z = t->z; v.q = t->q;
    v.xq = t->xq;
    v.xl = t->xq ? t->xq + t->xq_n4 : nullptr;
    v.perm = t->perm;
#if defined(DAFMM_CHECK)
    v.n = t->n;
    v.nrec = (int64_t)t->xq_n4;
    v.nu = t->nu;
    v.nw = t->nw;
    v.nx = t->nx;
#endif
    return v;
}

// per-box arrays of the adaptive hierarchy, sized for `cap` boxes (ints per box)
constexpr int kBoxArrays = 8;
constexpr size_t kBoxWidth[kBoxArrays] = {1, 1, 3, 1, 8, 1, 1, 27};  // root level ijk parent child pbeg pend colleague
constexpr size_t kBoxInts = 43;

int** box_array(dafmm_tree* t, int k) {
    int** a[kBoxArrays] = {&t->a_root, &t->a_level, &t->a_ijk, &t->a_parent, &t->a_child, &t->a_pbeg, &t->a_pend,
                           &t->a_colleague};
    return a[k];
}

void free_box_arrays(dafmm_ctx* c, dafmm_tree* t) {
    for (int k = 0; k < kBoxArrays; ++k) {
        dev_free(c, *box_array(t, k), (size_t)t->cap * kBoxWidth[k] * 4);
        *box_array(t, k) = nullptr;
    }
    t->cap = 0;
}

// grow the box arrays to hold `need` boxes, keeping the first `used`
int grow_boxes(dafmm_ctx* c, dafmm_tree* t, int need, int used, cudaStream_t s) {
    if (need <= t->cap) return DAFMM_OK;
    int cap = t->cap ? t->cap : 1024;
    while (cap < need) cap *= 2;
    int* nb[kBoxArrays] = {};
    for (int k = 0; k < kBoxArrays; ++k) {
        int rc = dev_alloc(c, (void**)&nb[k], (size_t)cap * kBoxWidth[k] * 4, "tree boxes");
        if (rc) {
            for (int j = 0; j < k; ++j) dev_free(c, nb[j], (size_t)cap * kBoxWidth[j] * 4);
            return rc;
        }
        int* old = *box_array(t, k);
        if (used && old)
            CK(c, cudaMemcpyAsync(nb[k], old, (size_t)used * kBoxWidth[k] * 4, cudaMemcpyDeviceToDevice, s), "grow");
    }
    CK(c, cudaStreamSynchronize(s), "grow");
    free_box_arrays(c, t);
    for (int k = 0; k < kBoxArrays; ++k) *box_array(t, k) = nb[k];
    t->cap = cap;
    return DAFMM_OK;
}

void free_adaptive(dafmm_ctx* c, dafmm_tree* t) {
    free_box_arrays(c, t);
    dev_free(c, t->aLh, t->aLh_bytes);
    t->aLh = nullptr;
    t->aLh_bytes = 0;
    dev_free(c, t->aMc, t->aMc_bytes);
    t->aMc = nullptr;
    t->aMc_bytes = 0;
    const size_t nb1 = (size_t)t->nbox + 1;
    dev_free(c, t->a_geom, (size_t)t->nbox * sizeof(double4));
    dev_free(c, t->a_xq0, (size_t)t->nbox * sizeof(int));
    t->a_xq0 = nullptr;
    dev_free(c, t->d_rootdom, t->rootdom.size() * sizeof(double));
    dev_free(c, t->u_ptr, nb1 * 4); dev_free(c, t->w_ptr, nb1 * 4); dev_free(c, t->x_ptr, nb1 * 4);
    dev_free(c, t->u_idx, (size_t)t->nu * 4); dev_free(c, t->w_idx, (size_t)t->nw * 4); dev_free(c, t->x_idx, (size_t)t->nx * 4);
    dev_free(c, t->leaves, (size_t)t->nleaves * 4);
    dev_free(c, t->grp_tg, (size_t)t->nbox * 4);
    dev_free(c, t->grp_ptr, ((size_t)(t->maxlev + 1) * 8 + 1) * 4);
    if (t->a_exp_p >= 0) {
        const size_t cnt = (size_t)t->nbox * ncp_of(t->a_exp_p);
        dev_free(c, t->aM, cnt * 8); dev_free(c, t->aL, cnt * 8); dev_free(c, t->aMf, cnt * 8);
    }
    t->u_ptr = t->w_ptr = t->x_ptr = t->u_idx = t->w_idx = t->x_idx = t->leaves = t->grp_tg = t->grp_ptr = nullptr;
    dev_free(c, t->aMinv, (size_t)t->nbox * sizeof(float));
    t->aMinv = nullptr;
    t->a_geom = nullptr;
    t->d_rootdom = nullptr;
    t->aM = t->aL = nullptr;
    t->aMf = nullptr;
    t->a_exp_p = -1;
}

// device scratch that is returned to the context when it goes out of scope
struct Scratch {
    dafmm_ctx* c;
    void* p = nullptr;
    size_t bytes = 0;
    explicit Scratch(dafmm_ctx* ctx) : c(ctx) {}
    int alloc(size_t b, const char* what) {
        release();
        bytes = b;
        return dev_alloc(c, &p, b, what);
    }
    void release() {
        dev_free(c, p, bytes);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
    ~Scratch() { release(); }
};

// root cubes of the trees: given, or the smallest cube around each tree's points, enlarged by
// 1e-12 of its size (the same rule as for a single tree)
int forest_domains(dafmm_ctx* c, const double* dxyz, const std::vector<int>& offs, const double* domains,
                   std::vector<double>& dom, const int* d_offs, cudaStream_t s) {
    const int nroots = (int)offs.size() - 1;
    dom.assign(4 * (size_t)nroots, 0.0);
    if (domains) {
        for (int r = 0; r < nroots; ++r) {
            const double* d = domains + 4 * r;
            if (!(d[3] > 0.0 && isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2]) && isfinite(d[3])))
                return fail(c, DAFMM_ERR_INVALID_ARG, "domain of tree " + std::to_string(r));
            for (int k = 0; k < 4; ++k) dom[4 * r + k] = d[k];
        }
        return DAFMM_OK;
    }
    Scratch bb(c);
    int rc = bb.alloc((size_t)nroots * 6 * 8, "bbox");
    if (rc) return rc;
    std::vector<unsigned long long> h(6 * (size_t)nroots);
    cudaError_t e = launch_bbox_roots(dxyz, d_offs, nroots, bb.as<unsigned long long>(), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), bb.p, h.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "bounding boxes");
    for (int r = 0; r < nroots; ++r) {
        double* d = &dom[4 * r];
        if (offs[r + 1] == offs[r]) {
            d[3] = 1.0;
            continue;
        }
        double v[6];
        for (int k = 0; k < 6; ++k) {
            unsigned long long u = h[6 * r + k];
            u = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
            memcpy(&v[k], &u, 8);
        }
        double size = std::max(v[3] - v[0], std::max(v[4] - v[1], v[5] - v[2]));
        if (!(size > 0.0)) size = 1.0;
        size = size * (1.0 + 1e-12);
        if (!(isfinite(size) && isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2])))
            return fail(c, DAFMM_ERR_INVALID_ARG, "non-finite coordinates");
        d[0] = v[0]; d[1] = v[1]; d[2] = v[2]; d[3] = size;
    }
    return DAFMM_OK;
}

// keys -> sort (-> regroup by tree) -> level-by-level split -> colleagues -> geometry ->
// leaves -> gather -> U, W, X lists -> M2L target groups.  t->rootdom holds the root cubes.
int build_adaptive(dafmm_ctx* c, dafmm_tree* t, const double* dxyz, const double* dq, const std::vector<int>& offs,
                   const int* d_offs, int max_leaf, int max_depth, cudaStream_t s) {
    const int64_t n = t->n;
    const size_t N1 = (size_t)(n > 0 ? n : 1);
    const int nroots = (int)offs.size() - 1;
    int rc;
    cudaError_t e;
    Scratch keys(c), tmp(c), scratch(c);
    if ((rc = keys.alloc(N1 * 8, "sort keys"))) return rc;
    if ((rc = tmp.alloc(radix_sort_temp_bytes(n > 0 ? n : 1), "sort scratch"))) return rc;
    if ((rc = dev_alloc(c, (void**)&t->d_rootdom, t->rootdom.size() * sizeof(double), "root cubes"))) return rc;
    CK(c, cudaMemcpyAsync(t->d_rootdom, t->rootdom.data(), t->rootdom.size() * sizeof(double), cudaMemcpyHostToDevice,
                          s), "root cubes");
    e = launch_morton_keys(dxyz, n, d_offs, nroots, t->d_rootdom, keys.as<uint64_t>(), t->perm, s);
    if (e == cudaSuccess) e = radix_sort_pairs(keys.as<uint64_t>(), t->perm, n, 3 * kQBits, tmp.p, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Morton sort");
    if (nroots > 1 && n > 0) {
        // stable regroup by tree: sort positions by tree index, then apply to (perm, keys)
        Scratch tk(c), pos(c), perm2(c), keys2(c);
        if ((rc = tk.alloc(N1 * 8, "tree keys")) || (rc = pos.alloc(N1 * 4, "tree keys")) ||
            (rc = perm2.alloc(N1 * 4, "tree keys")) || (rc = keys2.alloc(N1 * 8, "tree keys")))
            return rc;
        int bits = 1;
        while ((1 << bits) < nroots) ++bits;
        e = launch_tree_keys(t->perm, n, d_offs, nroots, tk.as<uint64_t>(), pos.as<int>(), s);
        if (e == cudaSuccess) e = radix_sort_pairs(tk.as<uint64_t>(), pos.as<int>(), n, bits, tmp.p, s);
        if (e == cudaSuccess)
            e = launch_apply_order(pos.as<int>(), n, t->perm, keys.as<uint64_t>(), perm2.as<int>(),
                                   keys2.as<uint64_t>(), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(t->perm, perm2.p, N1 * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(keys.p, keys2.p, N1 * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "tree regroup");
    }
    // roots
    if ((rc = grow_boxes(c, t, std::max(1024, nroots), 0, s))) return rc;
    {
        std::vector<int> zero(3 * (size_t)nroots, 0), m1(nroots, -1), lev(nroots, 0), rid(nroots), pb(nroots),
            pe(nroots);
        for (int r = 0; r < nroots; ++r) {
            rid[r] = r;
            pb[r] = offs[r];
            pe[r] = offs[r + 1];
        }
        const size_t R = (size_t)nroots * 4;
        CK(c, cudaMemcpyAsync(t->a_root, rid.data(), R, cudaMemcpyHostToDevice, s), "roots");
        CK(c, cudaMemcpyAsync(t->a_level, lev.data(), R, cudaMemcpyHostToDevice, s), "roots");
        CK(c, cudaMemcpyAsync(t->a_ijk, zero.data(), 3 * R, cudaMemcpyHostToDevice, s), "roots");
        CK(c, cudaMemcpyAsync(t->a_parent, m1.data(), R, cudaMemcpyHostToDevice, s), "roots");
        CK(c, cudaMemcpyAsync(t->a_pbeg, pb.data(), R, cudaMemcpyHostToDevice, s), "roots");
        CK(c, cudaMemcpyAsync(t->a_pend, pe.data(), R, cudaMemcpyHostToDevice, s), "roots");
        CK(c, cudaStreamSynchronize(s), "roots");
    }
    t->level_start.assign({0, nroots});
    for (int l = 0; l < max_depth; ++l) {
        const int lb = t->level_start[l], le = t->level_start[l + 1];
        const int nl = le - lb;
        if (scratch.bytes < 2 * ((size_t)nl + 1) * 4 && (rc = scratch.alloc(2 * ((size_t)nl + 1) * 4, "split scratch")))
            return rc;
        int* cnt = scratch.as<int>();
        int* off = cnt + nl + 1;
        e = launch_split(abuild(t, keys.as<uint64_t>()), lb, le, l, max_leaf, max_depth, cnt, s);
        if (e == cudaSuccess) e = launch_scan(cnt, off, nl, s);
        int total = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, off + nl, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "split");
        if (total == 0) break;
        if ((rc = grow_boxes(c, t, le + total, le, s))) return rc;
        e = launch_split_fill(abuild(t, keys.as<uint64_t>()), lb, le, l, off, le, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "split");
        t->level_start.push_back(le + total);
    }
    t->maxlev = (int)t->level_start.size() - 2;
    t->nbox = t->level_start.back();
    const int nbox = t->nbox;
    e = launch_children_init(t->a_child, t->level_start[t->maxlev], nbox, s);
    for (int l = 0; l <= t->maxlev && e == cudaSuccess; ++l)
        e = launch_colleagues(abuild(t, keys.as<uint64_t>()), t->level_start[l], t->level_start[l + 1], s);
    if (e != cudaSuccess) return cuda_fail(c, e, "colleagues");
    if ((rc = dev_alloc(c, (void**)&t->a_geom, (size_t)nbox * sizeof(double4), "box geometry"))) return rc;
    e = launch_box_geometry(t->a_root, t->a_level, t->a_ijk, t->d_rootdom, nbox, t->a_geom, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "geometry");
    // leaves (breadth-first order)
    if ((rc = scratch.alloc(2 * ((size_t)nbox + 1) * 4, "leaf scratch"))) return rc;
    int* flags = scratch.as<int>();
    int* foff = flags + nbox + 1;
    e = launch_leaf_flags(t->a_child, nbox, flags, s);
    if (e == cudaSuccess) e = launch_scan(flags, foff, nbox, s);
    int nl = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nl, foff + nbox, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "leaves");
    t->nleaves = nl;
    if ((rc = dev_alloc(c, (void**)&t->leaves, (size_t)(nl > 0 ? nl : 1) * 4, "leaves"))) return rc;
    e = launch_scatter_flagged(flags, foff, nbox, t->leaves, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "leaves");
    // FP32 records: leaves in list order take consecutive even record ranges (at most one
    // padding record per leaf)
    dev_free(c, t->xq, 2 * t->xq_n4 * sizeof(float4));
    t->xq = nullptr;
    t->xq_n4 = xq_records(t->n, nl);
    if ((rc = dev_alloc(c, (void**)&t->xq, 2 * t->xq_n4 * sizeof(float4), "particles"))) {
        t->xq_n4 = 0;
        return rc;
    }
    if ((rc = dev_alloc(c, (void**)&t->a_xq0, (size_t)nbox * sizeof(int), "leaf records"))) return rc;
    CK(c, cudaMemsetAsync(t->a_xq0, 0, (size_t)nbox * sizeof(int), s), "memset");
    e = launch_leaf_records(t->leaves, nl, t->a_pbeg, t->a_pend, flags, foff, t->a_xq0, s);
    if (e == cudaSuccess)
        e = launch_gather_adaptive(dxyz, dq, t->perm, abuild(t, keys.as<uint64_t>()), t->leaves, nl, t->a_geom,
                                   t->a_xq0, t->x, t->y, t->z, t->q, t->xq, t->xq_n4, t->n, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "gather");
    // U, W, X lists
    const size_t nb1 = (size_t)nbox + 1;
    Scratch cnt3(c);
    if ((rc = cnt3.alloc(3 * nb1 * 4 + 32, "list counts"))) return rc;
    int* cu = cnt3.as<int>();
    unsigned long long* nv = reinterpret_cast<unsigned long long*>(cu + ((3 * nb1 + 1) & ~size_t(1)));
    // overflow of the list traversal, the tree build's own flag: the context's record of expired
    // device waits (read by dafmm_sync) must survive a tree build
    int* lflag = reinterpret_cast<int*>(nv + 1);
    if ((rc = dev_alloc(c, (void**)&t->u_ptr, nb1 * 4, "lists")) || (rc = dev_alloc(c, (void**)&t->w_ptr, nb1 * 4, "lists")) ||
        (rc = dev_alloc(c, (void**)&t->x_ptr, nb1 * 4, "lists")))
        return rc;
    CK(c, cudaMemsetAsync(nv, 0, 16, s), "counter");  // the V-pair counter and lflag
    e = launch_list_count(abuild(t, keys.as<uint64_t>()), nbox, cu, cu + nb1, cu + 2 * nb1, nv, lflag, s);
    if (e == cudaSuccess) e = launch_scan(cu, t->u_ptr, nbox, s);
    if (e == cudaSuccess) e = launch_scan(cu + nb1, t->w_ptr, nbox, s);
    if (e == cudaSuccess) e = launch_scan(cu + 2 * nb1, t->x_ptr, nbox, s);
    int tot[3] = {0, 0, 0};
    unsigned long long nvh = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[0], t->u_ptr + nbox, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[1], t->w_ptr + nbox, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[2], t->x_ptr + nbox, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nvh, nv, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "lists");
    t->nu = tot[0]; t->nw = tot[1]; t->nx = tot[2];
    t->nv = (int64_t)nvh;
    if ((rc = dev_alloc(c, (void**)&t->u_idx, (size_t)std::max(tot[0], 1) * 4, "lists")) ||
        (rc = dev_alloc(c, (void**)&t->w_idx, (size_t)std::max(tot[1], 1) * 4, "lists")) ||
        (rc = dev_alloc(c, (void**)&t->x_idx, (size_t)std::max(tot[2], 1) * 4, "lists")))
        return rc;
    e = launch_list_fill(abuild(t, keys.as<uint64_t>()), nbox, t->u_ptr, t->w_ptr, t->x_ptr, t->u_idx, t->w_idx,
                         t->x_idx, lflag, s);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, lflag, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "lists");
    if (flag) return fail(c, DAFMM_ERR_INVALID_ARG, "adaptive tree too deep for the list traversal");
    cnt3.release();
    // M2L target groups: boxes of levels >= 2 by (level, octant)
    const int ngroups = (t->maxlev + 1) * 8;
    {
        Scratch gk(c), gtmp(c);
        if ((rc = gk.alloc((size_t)nbox * 8, "groups")) || (rc = gtmp.alloc(radix_sort_temp_bytes(nbox), "groups")) ||
            (rc = dev_alloc(c, (void**)&t->grp_tg, (size_t)nbox * 4, "groups")) ||
            (rc = dev_alloc(c, (void**)&t->grp_ptr, ((size_t)ngroups + 1) * 4, "groups")))
            return rc;
        e = launch_group_keys(t->a_level, t->a_ijk, nbox, gk.as<uint64_t>(), t->grp_tg, s);
        if (e == cudaSuccess) e = radix_sort_pairs(gk.as<uint64_t>(), t->grp_tg, nbox, 8, gtmp.p, s);
        if (e == cudaSuccess) e = launch_group_ptr(gk.as<uint64_t>(), nbox, ngroups, t->grp_ptr, s);
        t->grp_ptr_h.assign(ngroups + 1, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t->grp_ptr_h.data(), t->grp_ptr, (ngroups + 1) * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "groups");
    }
    // largest leaf
    std::vector<int> pb(nbox), pe(nbox), lf(nl);
    CK(c, cudaMemcpy(pb.data(), t->a_pbeg, (size_t)nbox * 4, cudaMemcpyDeviceToHost), "info");
    CK(c, cudaMemcpy(pe.data(), t->a_pend, (size_t)nbox * 4, cudaMemcpyDeviceToHost), "info");
    CK(c, cudaMemcpy(lf.data(), t->leaves, (size_t)nl * 4, cudaMemcpyDeviceToHost), "info");
    for (int b : lf) t->max_per_leaf = std::max(t->max_per_leaf, pe[b] - pb[b]);
    return DAFMM_OK;
}

int ensure_adaptive_expansions(dafmm_tree* t, int p, cudaStream_t s) {
    if (t->a_exp_p == p) return DAFMM_OK;
    dafmm_ctx* c = t->ctx;
    if (t->a_exp_p >= 0) {
        const size_t cnt = (size_t)t->nbox * ncp_of(t->a_exp_p);
        dev_free(c, t->aM, cnt * 8); dev_free(c, t->aL, cnt * 8); dev_free(c, t->aMf, cnt * 8);
        t->a_exp_p = -1;
    }
    const size_t cnt = (size_t)t->nbox * ncp_of(p);
    int rc;
    if ((rc = dev_alloc(c, (void**)&t->aM, cnt * 8, "multipoles"))) return rc;
    if ((rc = dev_alloc(c, (void**)&t->aL, cnt * 8, "locals"))) return rc;
    // FP32 multipoles, or their TF32 high parts followed by the low parts
    if ((rc = dev_alloc(c, (void**)&t->aMf, cnt * 8, "multipoles (FP32)"))) return rc;
    if (!t->aMinv && (rc = dev_alloc(c, (void**)&t->aMinv, (size_t)t->nbox * sizeof(float), "multipole factors")))
        return rc;
    CK(c, cudaMemsetAsync(t->aM, 0, cnt * 8, s), "memset");
    CK(c, cudaMemsetAsync(t->aL, 0, cnt * 8, s), "memset");
    CK(c, cudaMemsetAsync(t->aMf, 0, cnt * 8, s), "memset");
    t->a_exp_p = p;
    return DAFMM_OK;
}

int eval_adaptive(dafmm_tree* t, int order, int precision, double* dphi, double* dfield, cudaStream_t s) {
    dafmm_ctx* c = t->ctx;
    const OrderOps* ops = order_ops(order);
    const bool far = t->maxlev >= 2;
    int rc;
    if ((rc = ensure_order(c, order, s, far))) return rc;
    if ((rc = ensure_adaptive_expansions(t, order, s))) return rc;
    const OrderData& od = c->ord[order];
    const AdaptiveView av = aview(t);
    auto mark = [&](int k) {
        if (c->profile) cudaEventRecord(c->ev[k], s);
    };
    int launches = 0;
    bool f32_locals = false;
    mark(0);
    if (far) {
        const size_t cnt = (size_t)t->nbox * od.ncp;
        const bool tc = precision != DAFMM_FP64 && c->m2l_kernel == 0 && c->tc_capable && order >= 2 &&
                        (precision != DAFMM_FP32 || (c->tc_mask & 1));
        const bool f16 = tc && precision == DAFMM_FP32 && c->m2l_f16;
        // the tensor-core M2L in the harmonic basis: (p + 1)^2 free coefficients per row (F16
        // operands in the FP32 mode, TF32 in MIXED); its output rows go to t->aLh
        const bool harm = tc && c->m2l_harm;
        // F16 split: hi and lo rows of rowlen16 halves (harmonic: rowlen16h), stored in the FP32
        // multipole buffer; TF32 split: hi and lo rows of ncp floats (harmonic: harm_row) there
        const size_t c16 = (size_t)t->nbox * (harm ? tc_rowlen16h(order) : tc_rowlen16(order));
        const size_t ctf = harm ? (size_t)t->nbox * harm_row(order) : cnt;
        void* h16 = t->aMf;
        void* l16 = reinterpret_cast<__half*>(t->aMf) + c16;
        if (harm) {
            const size_t need = (size_t)t->nbox * harm_row(order) * sizeof(float);
            if (t->aLh_bytes != need) {
                dev_free(c, t->aLh, t->aLh_bytes);
                t->aLh = nullptr;
                t->aLh_bytes = 0;
                if ((rc = dev_alloc(c, (void**)&t->aLh, need, "locals (harmonic)"))) return rc;
                t->aLh_bytes = need;
            }
            if ((rc = ensure_k16h(c, order, s))) return rc;
        }
        float* lh = t->aLh;
        // P2M and M2M in the harmonic basis too when the M2L is: free coefficients only (the
        // M2L reads nothing else); the others are filled in after the M2M, for the M2P
        const int prec_m = precision | (harm ? kRowsHarm : 0);
        CK(c, ops->p2m_a(av, t->leaves, t->nleaves, prec_m, t->aM, s), "P2M");
        ++launches;
        mark(1);
        for (int l = t->maxlev - 1; l >= 2; --l) {
            CK(c, ops->m2m_a(od, av, prec_m, t->level_start[l], t->level_start[l + 1], t->aM, s), "M2M");
            ++launches;
        }
        if (harm) {
            CK(c, harm_fill(order, t->aM, t->nbox, od.hx_step, od.hx_w64, od.hx_cst, s), "M2M (harmonic fill)");
            ++launches;
        }
        mark(2);
        if (f16) {
            if (!harm && (rc = ensure_k16(c, order, s))) return rc;
            const void* src = t->aM;
            const int nrows = t->nbox;
            float* inv = t->aMinv;
            CK(c, tc_split_f16_multi(1, &src, &nrows, &h16, &l16, &inv, order, s, false, harm), "split");
            ++launches;
        } else if (tc) {
            if (harm) CK(c, tc_split_tf32_harm(t->aM, t->nbox, order, t->aMf, t->aMf + ctf, s), "split");
            else CK(c, tc_split_tf32(t->aM, t->aMf, t->aMf + cnt, cnt, s), "split");
            ++launches;
        } else if (precision != DAFMM_FP64) {
            k_to_float<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 152 * 16), 256, 0, s>>>(t->aM, t->aMf, cnt);
            CK(c, cudaGetLastError(), "convert");
            ++launches;
        }
        mark(3);
        if (tc) {
            // every level in one launch of the gathered tensor-core contraction
            mark(4);
            TCGArgs a;
            memset(&a, 0, sizeof(a));
            a.f16 = f16;
            a.harm = harm;
            a.a_hi = f16 ? h16 : (const void*)t->aMf;
            a.a_lo = f16 ? l16 : (const void*)(t->aMf + ctf);
            a.a_inv = t->aMinv;
            a.b_hi = f16 ? (harm ? od.Kh16h : od.Kh16) : (const void*)(harm ? od.Khih : od.Khi);
            a.b_lo = f16 ? (harm ? od.Kl16h : od.Kl16) : (const void*)(harm ? od.Kloh : od.Klo);
            a.inv_r = harm ? od.k16h_inv_r : od.k16_inv_r;
            a.inv_c = harm ? od.k16h_inv_c : od.k16_inv_c;
            a.nkey = kNumKeys;
            a.tg = t->grp_tg;
            a.parent = t->a_parent;
            a.colleague = t->a_colleague;
            a.child = t->a_child;
            a.geom = t->a_geom;
            a.out = harm ? reinterpret_cast<double*>(lh) : t->aL;
            a.err = c->d_err;
            a.nbox = t->nbox;
            a.num_sms = c->num_sms;
            for (int l = t->maxlev; l >= 2; --l)  // finest first
                for (int o = 0; o < 8; ++o) {
                    a.grp_start[a.ngroups] = t->grp_ptr_h[l * 8 + o];
                    a.grp_count[a.ngroups] = t->grp_ptr_h[l * 8 + o + 1] - t->grp_ptr_h[l * 8 + o];
                    a.grp_oct[a.ngroups] = o;
                    ++a.ngroups;
                }
            CK(c, tcg_launch(order, a, s), "M2L (tensor cores)");
            ++launches;
            if (harm) {
                // the other coefficients of the locals of every box of levels >= 2 (the M2L's
                // targets, contiguous from level_start[2])
                const int b0 = t->level_start[2];
                const float* red = lh + (size_t)b0 * harm_row(order);
                void* full = t->aL + (size_t)b0 * od.ncp;
                const int nrows = t->nbox - b0;
                CK(c, tc_harm_expand(order, 1, &red, &full, nullptr, nullptr, &nrows, false, od.hx_step, od.hx_w,
                                     od.hx_cst, s),
                   "M2L (harmonic expansion)");
                ++launches;
            }
            for (int l = 2; l <= t->maxlev; ++l) {
                CK(c, ops->p2l_a(av, precision, t->level_start[l], t->level_start[l + 1], t->aL, s), "P2L");
                ++launches;
            }
        } else {
            // FP64: the M2L by rotation (Sec. 3.4), by default from p = 4
            const bool rot = precision == DAFMM_FP64 && (c->m2l_rot > 0 || (c->m2l_rot < 0 && order >= 4));
            if (rot && (rc = ensure_rotation(c, order, s))) return rc;
            const int rflags = rot ? kM2LRot | (c->m2l_harm ? kM2LHarm : 0) : 0;
            for (int l = 2; l <= t->maxlev; ++l) {
                if (l == t->maxlev) mark(4);
                int mx = 0;
                for (int o = 0; o < 8; ++o) mx = std::max(mx, t->grp_ptr_h[l * 8 + o + 1] - t->grp_ptr_h[l * 8 + o]);
                CK(c, ops->m2l_a(od, av, precision | rflags, t->grp_tg, t->grp_ptr, l * 8, mx, t->aM,
                                 t->aMf, t->aL, s),
                   "M2L");
                CK(c, ops->p2l_a(av, precision, t->level_start[l], t->level_start[l + 1], t->aL, s), "P2L");
                launches += 2;
            }
        }
        mark(5);
        for (int l = 2; l < t->maxlev; ++l) {  // parents at level l, children at l + 1
            CK(c, ops->l2l_a(od, av, precision, t->level_start[l], t->level_start[l + 1], t->aL, s), "L2L");
            ++launches;
        }
        mark(6);
    } else {
        for (int k = 1; k <= 6; ++k) mark(k);
    }
    // FP32 paths: the leaves' M2P reads FP32 multipole rows (no FP64 conversion per W box)
    float* mc = nullptr;
    if (far && precision != DAFMM_FP64) {
        const size_t cnt = (size_t)t->nbox * ncp_of(order);
        if (t->aMc_bytes != cnt * sizeof(float)) {
            dev_free(c, t->aMc, t->aMc_bytes);
            t->aMc = nullptr;
            t->aMc_bytes = 0;
            if ((rc = dev_alloc(c, (void**)&t->aMc, cnt * sizeof(float), "multipoles (FP32 copy)"))) return rc;
            t->aMc_bytes = cnt * sizeof(float);
        }
        k_to_float<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 152 * 16), 256, 0, s>>>(t->aM, t->aMc, cnt);
        CK(c, cudaGetLastError(), "convert");
        ++launches;
        mc = t->aMc;
    }
    CK(c, ops->leaf_a(av, t->leaves, t->nleaves, precision, t->aL, t->aM, mc, dphi, dfield, c->leaf_warps, s),
       "P2P/M2P/L2P");
    ++launches;
    mark(7);
    c->last_launches = launches;
    c->have_profile = c->profile;
    return DAFMM_OK;
}
}  // namespace

namespace dafmm {
const char* check_site_name(int site) {
    switch (site) {
        case kChkLeafRange: return "particle range of a uniform leaf";
        case kChkBoxIndex: return "box index from a tree array or list";
        case kChkBoxRange: return "particle range of an adaptive box";
        case kChkListPtr: return "interaction-list range";
        case kChkRotTask: return "rotation task entry";
        case kChkRecord: return "FP32 record of a leaf";
        case kChkSortScatter: return "radix-sort scatter position";
        case kChkPerm: return "sort permutation entry";
        case kChkLeafKey: return "leaf of a sorted key";
        case kChkSplitChild: return "child box of an adaptive split";
        case kChkListFill: return "interaction-list fill position";
        case kChkGatherSource: return "source box of the gathered M2L";
        case kChkDebug: return "deliberate failure of dafmm_debug_check";
    }
    return "unknown";
}

#if defined(DAFMM_CHECK)
static std::mutex& check_mutex() {
    static std::mutex m;
    return m;
}
static std::vector<CheckTake>& check_readers() {  // built on first use: registrations run at load time
    static std::vector<CheckTake> v;
    return v;
}
void check_register(CheckTake take) {
    std::lock_guard<std::mutex> g(check_mutex());
    check_readers().push_back(take);
}
int check_take_all(long long* index, long long* bound) {
    std::lock_guard<std::mutex> g(check_mutex());
    int first = 0;
    for (CheckTake take : check_readers()) {
        long long i = 0, n = 0;
        const int site = take(&i, &n);
        if (site && !first) {
            first = site;
            *index = i;
            *bound = n;
        }
    }
    return first;
}
#endif

int ctx_alloc(dafmm_ctx* c, void** p, size_t bytes, const char* what) { return dev_alloc(c, p, bytes, what); }
void ctx_free(dafmm_ctx* c, void* p, size_t bytes) { dev_free(c, p, bytes); }
}  // namespace dafmm

namespace dafmm {
const OrderOps* order_ops(int p) {
    switch (p) {
        case 0: return order_ops_p0();
        case 1: return order_ops_p1();
        case 2: return order_ops_p2();
        case 3: return order_ops_p3();
        case 4: return order_ops_p4();
        case 5: return order_ops_p5();
        case 6: return order_ops_p6();
        case 7: return order_ops_p7();
        case 8: return order_ops_p8();
        case 9: return order_ops_p9();
        case 10: return order_ops_p10();
    }
    return nullptr;
}
}  // namespace dafmm

int tree_ready(dafmm_tree* t, cudaStream_t s) {
    if (!t->built) return DAFMM_OK;
    dafmm_ctx* c = t->ctx;
    const cudaError_t q = cudaEventQuery(t->built);
    if (q == cudaErrorNotReady) {
        CK(c, cudaStreamWaitEvent(s, t->built, 0), "wait for the tree build");
        return DAFMM_OK;
    }
    // the build has ended: its scratch returns to the pool
    for (const auto& d : t->deferred) dev_free(c, d.first, d.second);
    t->deferred.clear();
    cudaEventDestroy(t->built);
    t->built = nullptr;
    return q == cudaSuccess ? DAFMM_OK : cuda_fail(c, q, "tree build");
}

// ================================ C ABI =======================================================
extern "C" {

int dafmm_create(dafmm_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return DAFMM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DAFMM_ERR_NO_DEVICE;
    }
    if (device < 0 || device >= ndev) return DAFMM_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return DAFMM_ERR_CUDA;
    dafmm_ctx* c = new dafmm_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return DAFMM_ERR_CUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    c->tc_capable = prop.major == 10;
    if (dev_alloc(c, (void**)&c->d_err, sizeof(int), "error flag") != DAFMM_OK ||
        cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        delete c;
        return DAFMM_ERR_CUDA;
    }
    *out = c;
    return DAFMM_OK;
}

int dafmm_create_pooled(dafmm_ctx** out, int device, size_t pool_bytes) {
    if (!out) return DAFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (pool_bytes < ((size_t)1 << 20)) return DAFMM_ERR_INVALID_ARG;
    dafmm_ctx* c = nullptr;
    int rc = dafmm_create(&c, device, pool_bytes);
    if (rc) return rc;
    pool_bytes = pool_bytes / OffsetArena::kAlign * OffsetArena::kAlign;
    cudaError_t e = cudaMalloc((void**)&c->arena_base, pool_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->arena_base = nullptr;
        dafmm_destroy(c);
        return DAFMM_ERR_OVER_BUDGET;
    }
    c->arena.reset(pool_bytes);
    *out = c;
    return DAFMM_OK;
}

void dafmm_destroy(dafmm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    std::vector<dafmm_tree*> ts = c->trees;
    for (dafmm_tree* t : ts) dafmm_tree_free(t);
    for (int p = 0; p <= kMaxOrder; ++p) free_order(c, c->ord[p]);
    for (int k = 0; k < 8; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    dev_free(c, c->d_err, sizeof(int));
    if (c->arena_base) cudaFree(c->arena_base);
    delete c;
}

const char* dafmm_last_error(const dafmm_ctx* c) { return c ? c->err.c_str() : "no context"; }

size_t dafmm_bytes_in_use(const dafmm_ctx* c) { return c ? c->in_use : 0; }

int dafmm_build_tree(dafmm_ctx* c, const double* xyz, const double* q, int64_t n, const double* domain,
                     int uniform_depth, int max_leaf, void* stream, dafmm_tree** out) {
    if (!c || !out) return DAFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || n > (int64_t)INT32_MAX - 1 || (n > 0 && (!xyz || !q)))
        return fail(c, DAFMM_ERR_INVALID_ARG, "particle arrays");
    if (uniform_depth < 0 && max_leaf < 1) return fail(c, DAFMM_ERR_INVALID_ARG, "max_leaf must be >= 1");
    if (uniform_depth > kMaxUniformDepth)
        return fail(c, DAFMM_ERR_INVALID_ARG, "uniform depth above " + std::to_string(kMaxUniformDepth));
    if (domain && !(domain[3] > 0.0 && isfinite(domain[0]) && isfinite(domain[1]) && isfinite(domain[2]) &&
                    isfinite(domain[3])))
        return fail(c, DAFMM_ERR_INVALID_ARG, "domain");
    CK(c, cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    Staged sx, sq;
    int rc;
    if ((rc = stage_in(c, xyz, (size_t)n * 3 * sizeof(double), s, sx))) return rc;
    if ((rc = stage_in(c, q, (size_t)n * sizeof(double), s, sq))) return rc;
    const double* dxyz = (const double*)sx.dev;
    const double* dq = (const double*)sq.dev;
    // a pooled context builds a uniform tree from host inputs asynchronously (below); the end
    // of the input copies is marked for it
    const bool async_build = c->arena_base && sx.owned && sq.owned && uniform_depth >= 0;
    if (async_build) {
        if (!c->ev_in) CK(c, cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming), "event");
        CK(c, cudaEventRecord(c->ev_in, s), "event");
    }

    dafmm_tree* t = new dafmm_tree();
    t->ctx = c;
    t->n = n;
    t->adaptive = uniform_depth < 0;
    t->max_leaf = max_leaf;
    t->depth = t->adaptive ? 0 : uniform_depth;
    t->nleaf = t->adaptive ? 0 : (int)level_boxes(uniform_depth);
    // root cube
    if (domain) {
        for (int d = 0; d < 4; ++d) t->dom[d] = domain[d];
    } else if (n > 0) {
        double* bb = nullptr;
        if ((rc = dev_alloc(c, (void**)&bb, 6 * sizeof(double), "bbox"))) { delete t; return rc; }
        cudaError_t e = launch_bbox(dxyz, n, bb, s);
        unsigned long long h[6];
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, bb, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dev_free(c, bb, 6 * sizeof(double));
        if (e != cudaSuccess) { delete t; return cuda_fail(c, e, "bounding box"); }
        double v[6];
        for (int k = 0; k < 6; ++k) {
            unsigned long long u = h[k];
            u = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
            memcpy(&v[k], &u, 8);
        }
        double size = std::max(v[3] - v[0], std::max(v[4] - v[1], v[5] - v[2]));
        if (!(size > 0.0)) size = 1.0;
        size = size * (1.0 + 1e-12);
        t->dom[0] = v[0]; t->dom[1] = v[1]; t->dom[2] = v[2]; t->dom[3] = size;
        if (!(isfinite(size) && isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]))) {
            delete t;
            return fail(c, DAFMM_ERR_INVALID_ARG, "non-finite coordinates");
        }
    }
    // device arrays
    const size_t N = (size_t)n;
    rc = 0;
    if (!rc) rc = dev_alloc(c, (void**)&t->x, N * sizeof(double), "particles");
    if (!rc) rc = dev_alloc(c, (void**)&t->y, N * sizeof(double), "particles");
    if (!rc) rc = dev_alloc(c, (void**)&t->z, N * sizeof(double), "particles");
    if (!rc) rc = dev_alloc(c, (void**)&t->q, N * sizeof(double), "particles");
    if (!rc) {
        t->xq_n4 = xq_records(n, t->nleaf);
        rc = dev_alloc(c, (void**)&t->xq, 2 * t->xq_n4 * sizeof(float4), "particles");
    }
    if (!rc) rc = dev_alloc(c, (void**)&t->perm, N * sizeof(int), "particles");
    if (!rc) rc = dev_alloc(c, (void**)&t->leaf_start, ((size_t)t->nleaf + 1) * sizeof(int), "leaves");
    if (t->adaptive) {
        if (rc) {
            c->trees.push_back(t);
            dafmm_tree_free(t);
            return rc;
        }
        c->trees.push_back(t);
        t->rootdom.assign(t->dom, t->dom + 4);
        t->root_offs = {0, n};
        const std::vector<int> offs = {0, (int)n};
        Scratch d_offs(c);
        if (!(rc = d_offs.alloc(2 * sizeof(int), "offsets"))) {
            const cudaError_t e =
                cudaMemcpyAsync(d_offs.p, offs.data(), 2 * sizeof(int), cudaMemcpyHostToDevice, s);
            rc = e != cudaSuccess ? cuda_fail(c, e, "offsets")
                                  : build_adaptive(c, t, dxyz, dq, offs, d_offs.as<int>(), max_leaf,
                                                   kMaxAdaptiveDepth, s);
        }
        if (rc) {
            dafmm_tree_free(t);  // a failed build leaves nothing behind in the context
            return rc;
        }
        *out = t;
        return DAFMM_OK;
    }
    uint64_t* keys = nullptr;
    void* tmp = nullptr;
    const size_t tmpb = radix_sort_temp_bytes(n);
    if (!rc) rc = dev_alloc(c, (void**)&keys, N * sizeof(uint64_t), "sort keys");
    if (!rc) rc = dev_alloc(c, &tmp, tmpb, "sort scratch");
    if (rc) {
        dev_free(c, keys, N * sizeof(uint64_t));
        dev_free(c, tmp, tmpb);
        c->trees.push_back(t);
        dafmm_tree_free(t);
        return rc;
    }
    const double scale = ldexp(1.0, kQBits) / t->dom[3];
    cudaError_t e = launch_uniform_keys(dxyz, n, t->dom[0], t->dom[1], t->dom[2], scale, t->depth, keys, t->perm, s);
    if (e == cudaSuccess) e = radix_sort_pairs(keys, t->perm, n, 3 * t->depth, tmp, s);
    if (e == cudaSuccess)
        e = launch_gather_uniform(dxyz, dq, t->perm, n, keys, make_view(t), t->x, t->y, t->z, t->q, t->xq,
                                  t->leaf_start, s);
    if (async_build && e == cudaSuccess) {
        // pooled context, host inputs (staged into the pool): the build stays in flight on its
        // stream.  An event marks its end (the tree's later users wait for it, tree_ready), its
        // scratch and staging go back to the pool once it has completed, and the largest leaf is
        // read back only when asked for.  The caller's host arrays may be reused once this
        // returns: their copies are waited for.
        e = cudaEventCreateWithFlags(&t->built, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(t->built, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(c->ev_in);
        if (e == cudaSuccess) {
            t->deferred.push_back({keys, N * sizeof(uint64_t)});
            t->deferred.push_back({tmp, tmpb});
            for (Staged* st : {&sx, &sq})
                if (st->owned) {
                    t->deferred.push_back({st->dev, st->bytes});
                    st->owned = false;
                }
            t->max_per_leaf = -1;
            c->trees.push_back(t);
            *out = t;
            return DAFMM_OK;
        }
        if (t->built) cudaEventDestroy(t->built);
        t->built = nullptr;
        cudaStreamSynchronize(s);  // nothing may still use the scratch freed below
    }
    // the largest leaf (for the caller's information)
    std::vector<int> ls((size_t)t->nleaf + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ls.data(), t->leaf_start, ls.size() * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(c, keys, N * sizeof(uint64_t));
    dev_free(c, tmp, tmpb);
    c->trees.push_back(t);
    if (e != cudaSuccess) {
        dafmm_tree_free(t);
        return cuda_fail(c, e, "tree build");
    }
    for (int b = 0; b < t->nleaf; ++b) t->max_per_leaf = std::max(t->max_per_leaf, ls[b + 1] - ls[b]);
    *out = t;
    return DAFMM_OK;
}

int dafmm_build_forest(dafmm_ctx* c, const double* xyz, const double* q, const int64_t* offsets, int ntrees,
                       const double* domains, int max_leaf, void* stream, dafmm_tree** out) {
    if (!c || !out) return DAFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (ntrees < 1 || !offsets || offsets[0] != 0) return fail(c, DAFMM_ERR_INVALID_ARG, "forest offsets");
    for (int r = 0; r < ntrees; ++r)
        if (offsets[r + 1] < offsets[r]) return fail(c, DAFMM_ERR_INVALID_ARG, "forest offsets decrease");
    const int64_t n = offsets[ntrees];
    if (n > (int64_t)INT32_MAX - 1 || (n > 0 && (!xyz || !q))) return fail(c, DAFMM_ERR_INVALID_ARG, "particle arrays");
    if (max_leaf < 1) return fail(c, DAFMM_ERR_INVALID_ARG, "max_leaf must be >= 1");
    CK(c, cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    Staged sx, sq;
    int rc;
    if ((rc = stage_in(c, xyz, (size_t)n * 3 * sizeof(double), s, sx))) return rc;
    if ((rc = stage_in(c, q, (size_t)n * sizeof(double), s, sq))) return rc;
    const double* dxyz = (const double*)sx.dev;
    const double* dq = (const double*)sq.dev;
    std::vector<int> offs(ntrees + 1);
    for (int r = 0; r <= ntrees; ++r) offs[r] = (int)offsets[r];
    Scratch d_offs(c);
    if ((rc = d_offs.alloc(offs.size() * sizeof(int), "forest offsets"))) return rc;
    CK(c, cudaMemcpyAsync(d_offs.p, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice, s), "offsets");
    dafmm_tree* t = new dafmm_tree();
    t->ctx = c;
    t->n = n;
    t->adaptive = true;
    t->max_leaf = max_leaf;
    t->depth = 0;
    t->nleaf = 0;
    t->nroots = ntrees;
    t->root_offs.assign(offsets, offsets + ntrees + 1);
    c->trees.push_back(t);
    rc = forest_domains(c, dxyz, offs, domains, t->rootdom, d_offs.as<int>(), s);
    if (!rc) {
        for (int d = 0; d < 4; ++d) t->dom[d] = t->rootdom[d];
        const size_t N = (size_t)n;
        if (!rc) rc = dev_alloc(c, (void**)&t->x, N * sizeof(double), "particles");
        if (!rc) rc = dev_alloc(c, (void**)&t->y, N * sizeof(double), "particles");
        if (!rc) rc = dev_alloc(c, (void**)&t->z, N * sizeof(double), "particles");
        if (!rc) rc = dev_alloc(c, (void**)&t->q, N * sizeof(double), "particles");
        if (!rc) rc = dev_alloc(c, (void**)&t->perm, N * sizeof(int), "particles");
        if (!rc) rc = dev_alloc(c, (void**)&t->leaf_start, sizeof(int), "leaves");
    }
    if (!rc) rc = build_adaptive(c, t, dxyz, dq, offs, d_offs.as<int>(), max_leaf, kMaxAdaptiveDepth, s);
    if (rc) {
        const std::string msg = c->err;
        dafmm_tree_free(t);
        c->err = msg;
        return rc;
    }
    *out = t;
    return DAFMM_OK;
}

int dafmm_forest_info(const dafmm_tree* t, int* ntrees, double* domains) {
    if (!t) return DAFMM_ERR_INVALID_ARG;
    if (ntrees) *ntrees = t->adaptive ? t->nroots : 1;
    if (domains) {
        if (t->adaptive)
            for (size_t k = 0; k < t->rootdom.size(); ++k) domains[k] = t->rootdom[k];
        else
            for (int d = 0; d < 4; ++d) domains[d] = t->dom[d];
    }
    return DAFMM_OK;
}

int dafmm_tree_free(dafmm_tree* t) {
    if (!t) return DAFMM_ERR_INVALID_ARG;
    dafmm_ctx* c = t->ctx;
    cudaSetDevice(c->device);
    // (the work that uses the tree, its build included, has completed: the caller's contract)
    for (const auto& d : t->deferred) dev_free(c, d.first, d.second);
    t->deferred.clear();
    if (t->built) cudaEventDestroy(t->built);
    t->built = nullptr;
    free_expansions(t);
    const size_t N = (size_t)t->n;
    dev_free(c, t->x, N * sizeof(double));
    dev_free(c, t->y, N * sizeof(double));
    dev_free(c, t->z, N * sizeof(double));
    dev_free(c, t->q, N * sizeof(double));
    dev_free(c, t->xq, 2 * t->xq_n4 * sizeof(float4));
    dev_free(c, t->perm, N * sizeof(int));
    dev_free(c, t->leaf_start, ((size_t)t->nleaf + 1) * sizeof(int));
    dev_free(c, t->out_scratch, t->out_scratch_bytes);
    if (t->adaptive) free_adaptive(c, t);
    auto it = std::find(c->trees.begin(), c->trees.end(), t);
    if (it != c->trees.end()) c->trees.erase(it);
    delete t;
    return DAFMM_OK;
}

int dafmm_tree_info(const dafmm_tree* t, int64_t* info, double* domain4) {
    if (!t || !info) return DAFMM_ERR_INVALID_ARG;
    int64_t m2l = 0, p2p = 0;
    for (int l = 2; l <= t->depth; ++l) {
        const int64_t s = (int64_t)1 << l;
        // per axis: number of ordered (target, source) index pairs with |dt - ds| <= 1 among
        // children of adjacent parents, minus adjacent ones
        int64_t near1 = 3 * s - 2;  // pairs at distance <= 1
        int64_t par = 3 * (s / 2) - 2;  // adjacent parent pairs
        int64_t cand = par * 4;          // children pairs of adjacent parents
        m2l += cand * cand * cand - near1 * near1 * near1;
    }
    {
        const int64_t s = (int64_t)1 << t->depth;
        const int64_t near1 = 3 * s - 2;
        p2p = near1 * near1 * near1;
    }
    if (t->adaptive) {
        info[0] = t->n;
        info[1] = t->maxlev;
        info[2] = t->nleaves;
        info[3] = t->nbox;
        info[4] = t->max_per_leaf;
        info[5] = 1;
        info[6] = t->nv;
        info[7] = t->nu;
        if (domain4)
            for (int d = 0; d < 4; ++d) domain4[d] = t->dom[d];
        return DAFMM_OK;
    }
    if (t->max_per_leaf < 0) {  // the asynchronous build's largest leaf, read back once
        dafmm_tree* tm = const_cast<dafmm_tree*>(t);
        if (cudaSetDevice(t->ctx->device) != cudaSuccess || (t->built && cudaEventSynchronize(t->built) != cudaSuccess))
            return DAFMM_ERR_CUDA;
        std::vector<int> ls((size_t)t->nleaf + 1);
        if (cudaMemcpy(ls.data(), t->leaf_start, ls.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return DAFMM_ERR_CUDA;
        int mx = 0;
        for (int b = 0; b < t->nleaf; ++b) mx = std::max(mx, ls[b + 1] - ls[b]);
        tm->max_per_leaf = mx;
    }
    info[0] = t->n;
    info[1] = t->depth;
    info[2] = t->nleaf;
    int64_t nb = 0;
    for (int l = 0; l <= t->depth; ++l) nb += (int64_t)level_boxes(l);
    info[3] = nb;
    info[4] = t->max_per_leaf;
    info[5] = 0;
    info[6] = m2l;
    info[7] = p2p;
    if (domain4)
        for (int d = 0; d < 4; ++d) domain4[d] = t->dom[d];
    return DAFMM_OK;
}

int dafmm_eval(dafmm_tree* t, int order, double theta, int precision, double* phi, double* field, void* stream) {
    if (!t) return DAFMM_ERR_INVALID_ARG;
    dafmm_ctx* c = t->ctx;
    if (order < 0 || order > kMaxOrder) return fail(c, DAFMM_ERR_UNSUPPORTED_ORDER, std::to_string(order));
    if (!(fabs(theta - 1.0) < 1e-12))
        return fail(c, DAFMM_ERR_UNSUPPORTED, "theta other than 1 (nearest-neighbour separation)");
    if (precision != DAFMM_FP64 && precision != DAFMM_MIXED && precision != DAFMM_FP32 && precision != DAFMM_FF)
        return fail(c, DAFMM_ERR_INVALID_ARG, "precision");
    CK(c, cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = tree_ready(t, s))) return rc;
    if (t->n == 0) return DAFMM_OK;
    const OrderOps* ops = order_ops(order);
    const bool far = t->depth >= 2;
    if ((rc = ensure_order(c, order, s, far))) return rc;
    if (far && (rc = ensure_expansions(t, order, s))) return rc;
    // outputs
    const bool phi_dev = !phi || is_device_ptr(phi), field_dev = !field || is_device_ptr(field);
    double* dphi = phi;
    double* dfield = field;
    const size_t N = (size_t)t->n;
    if (!phi_dev || !field_dev) {
        const size_t need = N * 4 * sizeof(double);
        if (t->out_scratch_bytes < need) {
            dev_free(c, t->out_scratch, t->out_scratch_bytes);
            t->out_scratch = nullptr;
            t->out_scratch_bytes = 0;
            if ((rc = dev_alloc(c, (void**)&t->out_scratch, need, "output staging"))) return rc;
            t->out_scratch_bytes = need;
        }
        if (!phi_dev) dphi = t->out_scratch;
        if (!field_dev) dfield = t->out_scratch + N;
    }
    if (t->adaptive) {
        // (the float-float kernels serve uniform trees; adaptive trees take the FP64 path)
        if ((rc = eval_adaptive(t, order, precision == DAFMM_FF ? DAFMM_FP64 : precision, dphi, dfield, s))) return rc;
        if (!phi_dev) CK(c, cudaMemcpyAsync(phi, dphi, N * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (!field_dev) CK(c, cudaMemcpyAsync(field, dfield, N * 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
        if (!phi_dev || !field_dev) CK(c, cudaStreamSynchronize(s), "sync");
        return DAFMM_OK;
    }
    const TreeView tv = make_view(t);
    const OrderData& od = c->ord[order];
    const int L = t->depth;
    // phase boundaries: 0 start, 1 after P2M, 2 after M2M, 3 after conversions, 4 before the
    // finest M2L, 5 after M2L, 6 after L2L, 7 after L2P/P2P
    auto mark = [&](int k) {
        if (c->profile) cudaEventRecord(c->ev[k], s);
    };
    int launches = 0;
    bool f32_locals = false;
    mark(0);
    if (far) {
        const bool tc_ok = c->m2l_kernel == 0 && c->tc_capable && order >= 2;
        const bool f32 = precision == DAFMM_FP32;
        const bool fff = precision == DAFMM_FF;  // float-float P2M, M2L and leaves; FP64 shifts
        const bool tc_m2l = precision != DAFMM_FP64 && !fff && tc_ok && (!f32 || (c->tc_mask & 1));
        const bool tc_m2m = f32 && tc_ok && (c->tc_mask & 2);     // tensor-core M2M (FP32 mode)
        const bool tc_l2l = f32 && tc_ok && (c->tc_mask & 4);     // tensor-core L2L (FP32 mode)
        const bool f16_m2l = tc_m2l && f32 && c->m2l_f16;         // M2L on F16 split operands
        // FP32 mode with M2L and L2L on tensor cores keeps the locals as FP32 rows (in the
        // FP64 arrays' memory): the epilogues then need no FP64 arithmetic.  With the F16 M2L
        // and the SIMT M2M the multipoles are FP32 rows as well (P2M, M2M and the F16 split
        // all in FP32).
        f32_locals = tc_m2l && tc_l2l;
        const bool f32_mult = f16_m2l && !tc_m2m;
        Expansions& ex = t->ex;
        ex.M_f32 = f32_mult;
        // the tensor-core M2L in the harmonic basis: (p + 1)^2 free coefficients per row instead
        // of ncoef (F16 operands in the FP32 mode, TF32 in MIXED)
        const bool harm = tc_m2l && c->m2l_harm && (f16_m2l || !tc_m2m);  // (the tensor-core M2M
                                                                           // writes full TF32 rows)
        // ... and then P2M and M2M in it too: the M2L reads only the multipoles' free
        // coefficients, so only those are computed (the SIMT M2M; P2M in FP32)
        const bool harm_m = harm && !tc_m2m;
        ex.M_harm = harm_m;
        const int prec_m = precision | (f32_mult ? kRowsF32 : 0) | (harm_m ? kRowsHarm : 0);
        if (f16_m2l && (rc = ensure_f16_levels(t, s))) return rc;
        if (harm && ((rc = ensure_lh_levels(t)) || (rc = ensure_k16h(c, order, s)))) return rc;
        if (f16_m2l && !harm && (rc = ensure_k16(c, order, s))) return rc;
        auto tc_args = [&](int mode, int lmin, int lmax) {
            TCArgs a;
            memset(&a, 0, sizeof(a));
            a.mode = mode;
            a.lmin = lmin;
            a.lmax = lmax;
            a.err = c->d_err;
            a.num_sms = c->num_sms;
            return a;
        };
        // the FP32 harmonic P2M also writes the finest level's F16 split (its warp holds each row)
        const bool p2m_f16 = f16_m2l && f32_mult && harm_m;
        F16Rows fr;
        if (p2m_f16) {
            fr.hi = ex.Mh16[L];
            fr.lo = ex.Ml16[L];
            fr.inv = ex.Minv[L];
            fr.rowlen = tc_rowlen16h(order);
        }
        CK(c, ops->p2m(tv, prec_m, ex.M[L], p2m_f16 ? &fr : nullptr, s), "P2M");
        ++launches;
        mark(1);
        if (tc_m2m) {
            CK(c, tc_split_tf32(ex.M[L], ex.Mhi[L], ex.Mlo[L], level_boxes(L) * od.ncp, s), "split");
            ++launches;
            for (int lc = L; lc >= 3; --lc) {
                TCArgs a = tc_args(kTcM2M, lc, lc);
                a.a_hi[lc] = ex.Mhi[lc];
                a.a_lo[lc] = ex.Mlo[lc];
                a.out[lc] = ex.M[lc - 1];
                a.out_hi[lc] = ex.Mhi[lc - 1];
                a.out_lo[lc] = ex.Mlo[lc - 1];
                a.scale[lc] = 1.0;
                a.b_hi = od.M2Mhi;
                a.b_lo = od.M2Mlo;
                a.nkey = 8;
                CK(c, tc_launch(order, a, s), "M2M (tensor cores)");
                ++launches;
            }
        } else {
            for (int lc = L; lc >= 3; --lc) {
                CK(c, ops->m2m_level(od, prec_m, lc, ex.M[lc], ex.M[lc - 1], s), "M2M");
                ++launches;
            }
        }
        mark(2);
        if (f16_m2l) {
            const void* src[8];
            int nrows[8];
            void *hi[8], *lo[8];
            float* inv[8];
            const int lsplit = p2m_f16 ? L - 1 : L;  // (the P2M split the finest level)
            for (int l = 2; l <= lsplit; ++l) {
                src[l - 2] = ex.M[l];
                nrows[l - 2] = (int)level_boxes(l);
                hi[l - 2] = ex.Mh16[l];
                lo[l - 2] = ex.Ml16[l];
                inv[l - 2] = ex.Minv[l];
            }
            if (lsplit >= 2) {
                CK(c, tc_split_f16_multi(lsplit - 1, src, nrows, hi, lo, inv, order, s, f32_mult, harm), "split");
                ++launches;
            }
        } else if (precision != DAFMM_FP64 && !fff && !(tc_m2m && tc_m2l))
            for (int l = 2; l <= L; ++l) {
                const size_t cnt = level_boxes(l) * od.ncp;
                if (harm) {
                    CK(c, tc_split_tf32_harm(ex.M[l], level_boxes(l), order, ex.Mhi[l], ex.Mlo[l], s), "split");
                } else if (tc_m2l) {
                    CK(c, tc_split_tf32(ex.M[l], ex.Mhi[l], ex.Mlo[l], cnt, s), "split");
                } else {
                    k_to_float<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 152 * 16), 256, 0, s>>>(ex.M[l], ex.Mf[l], cnt);
                    CK(c, cudaGetLastError(), "convert");
                }
                ++launches;
            }
        mark(3);
        if (tc_m2l) {
            mark(4);
            TCArgs a = tc_args(kTcM2L, 2, L);
            a.f16 = f16_m2l;
            a.harm = harm;
            a.out_f32 = f32_locals || harm;
            for (int l = 2; l <= L; ++l) {
                a.a_hi[l] = f16_m2l ? ex.Mh16[l] : (const void*)ex.Mhi[l];
                a.a_lo[l] = f16_m2l ? ex.Ml16[l] : (const void*)ex.Mlo[l];
                a.a_inv[l] = ex.Minv[l];
                // harmonic basis: the free coefficients (FP32 rows), expanded below
                a.out[l] = harm ? reinterpret_cast<double*>(ex.Lh[l]) : ex.L[l];
                // the L2L of level 3 reads the TF32 split of level 2's locals; every finer
                // level's split is written by the L2L that completes it
                if (tc_l2l && l == 2 && !harm) {
                    a.out_hi[l] = ex.Lhi[l];
                    a.out_lo[l] = ex.Llo[l];
                }
                a.scale[l] = 1.0 / ldexp(t->dom[3], -l);
            }
            a.b_hi = f16_m2l ? (harm ? od.Kh16h : od.Kh16) : (const void*)(harm ? od.Khih : od.Khi);
            a.b_lo = f16_m2l ? (harm ? od.Kl16h : od.Kl16) : (const void*)(harm ? od.Kloh : od.Klo);
            a.inv_r = harm ? od.k16h_inv_r : od.k16_inv_r;
            a.inv_c = harm ? od.k16h_inv_c : od.k16_inv_c;
            a.nkey = kNumKeys;
            CK(c, tc_launch(order, a, s), "M2L (tensor cores)");
            ++launches;
            if (harm) {
                // every coefficient of the locals from the free ones (and the TF32 split of
                // level 2's, which the L2L of level 3 reads)
                const float* red[kTcMaxLevels];
                void* full[kTcMaxLevels];
                float *hs[kTcMaxLevels], *ls[kTcMaxLevels];
                int nrows[kTcMaxLevels];
                for (int l = 2; l <= L; ++l) {
                    red[l - 2] = ex.Lh[l];
                    full[l - 2] = ex.L[l];
                    hs[l - 2] = tc_l2l && l == 2 ? ex.Lhi[l] : nullptr;
                    ls[l - 2] = tc_l2l && l == 2 ? ex.Llo[l] : nullptr;
                    nrows[l - 2] = (int)level_boxes(l);
                }
                CK(c, tc_harm_expand(order, L - 1, red, full, hs, ls, nrows, f32_locals, od.hx_step, od.hx_w, od.hx_cst, s),
                   "M2L (harmonic expansion)");
                ++launches;
            }
        } else {
            // M2L by rotation (Sec. 3.4); by default from p = 4, where it is the faster one (FP64),
            // and from p = 2 in float-float
            const bool rot = precision == DAFMM_FP64 && (c->m2l_rot > 0 || (c->m2l_rot < 0 && order >= 4));
            const bool rot_ff = fff && order >= 2;
            if (rot && (rc = ensure_rotation(c, order, s))) return rc;
            if (rot_ff && (rc = ensure_rotation_ff(c, order, s))) return rc;
            for (int l = 2; l <= L; ++l) {
                if (l == L) mark(4);
                const double inv_h = 1.0 / ldexp(t->dom[3], -l);
                if (rot_ff) {
                    CK(c, ops->split_ff(ex.M[l], ex.Mhi[l], ex.Mlo[l], level_boxes(l) * od.ncp, s), "split");
                    CK(c, ops->m2l_rot_ff(od, l, ex.Mhi[l], ex.Mlo[l], ex.L[l], inv_h, c->m2l_harm != 0, s),
                       "M2L (rotation, float-float)");
                    ++launches;
                }
                else if (rot)
                    CK(c, ops->m2l_rot(od, l, ex.M[l], ex.L[l], inv_h, c->m2l_harm != 0, s), "M2L (rotation)");
                else
                    CK(c, ops->m2l_level(od, fff ? DAFMM_FP64 : precision, l, ex.M[l], ex.Mf[l], ex.L[l], inv_h, s),
                       "M2L");
                ++launches;
            }
        }
        mark(5);
        if (tc_l2l && !tc_m2l)  // the TF32 parts of the locals come from the tensor-core M2L otherwise
            for (int l = 2; l <= L; ++l) {
                CK(c, tc_split_tf32(ex.L[l], ex.Lhi[l], ex.Llo[l], level_boxes(l) * od.ncp, s), "split");
                ++launches;
            }
        for (int lc = 3; lc <= L; ++lc) {
            if (tc_l2l) {
                TCArgs a = tc_args(kTcL2L, lc, lc);
                a.out_f32 = f32_locals;
                a.a_hi[lc - 1] = ex.Lhi[lc - 1];
                a.a_lo[lc - 1] = ex.Llo[lc - 1];
                a.out[lc] = ex.L[lc];
                if (lc < L) {
                    a.out_hi[lc] = ex.Lhi[lc];
                    a.out_lo[lc] = ex.Llo[lc];
                }
                a.scale[lc] = 1.0;
                a.b_hi = od.L2Lhi;
                a.b_lo = od.L2Llo;
                a.nkey = 8;
                CK(c, tc_launch(order, a, s), "L2L (tensor cores)");
            } else {
                CK(c, ops->l2l_level(od, precision, lc, ex.L[lc - 1], ex.L[lc], s), "L2L");
            }
            ++launches;
        }
        mark(6);
    } else {
        for (int k = 1; k <= 6; ++k) mark(k);
    }
    TreeView tvl = tv;
    tvl.locals_f32 = f32_locals ? 1 : 0;
    if (far) t->ex.L_f32 = f32_locals;
    CK(c, ops->leaf(tvl, precision, far ? t->ex.L[L] : nullptr, dphi, dfield, s), "L2P/P2P");
    ++launches;
    mark(7);
    c->last_launches = launches;
    c->have_profile = c->profile;
    if (!phi_dev) CK(c, cudaMemcpyAsync(phi, dphi, N * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    if (!field_dev) CK(c, cudaMemcpyAsync(field, dfield, N * 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    if (!phi_dev || !field_dev) CK(c, cudaStreamSynchronize(s), "sync");
    return DAFMM_OK;
}

int dafmm_set_option(dafmm_ctx* c, int option, int64_t value) {
    if (!c) return DAFMM_ERR_INVALID_ARG;
    if (option == DAFMM_OPT_M2L_KERNEL && (value == 0 || value == 1)) {
        c->m2l_kernel = (int)value;
        return DAFMM_OK;
    }
    if (option == DAFMM_OPT_TC_MASK && value >= 0 && value <= 7) {
        c->tc_mask = (int)value;
        return DAFMM_OK;
    }
    if (option == DAFMM_OPT_LEAF_WARPS && (value == 1 || value == 2 || value == 4 || value == 8)) {
        c->leaf_warps = (int)value;
        return DAFMM_OK;
    }
    if (option == DAFMM_OPT_M2L_F16 && (value == 0 || value == 1)) {
        c->m2l_f16 = (int)value;
        return DAFMM_OK;
    }
    if (option == DAFMM_OPT_M2L_ROTATION && (value == -1 || value == 0 || value == 1)) {
        c->m2l_rot = (int)value;
        return DAFMM_OK;
    }
    if (option == DAFMM_OPT_M2L_HARMONIC && (value == 0 || value == 1)) {
        c->m2l_harm = (int)value;
        return DAFMM_OK;
    }
    return fail(c, DAFMM_ERR_INVALID_ARG, "option");
}

int dafmm_sync(dafmm_ctx* c, void* stream) {
    if (!c) return DAFMM_ERR_INVALID_ARG;
    CK(c, cudaSetDevice(c->device), "cudaSetDevice");
    CK(c, cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    int flag = 0;
    CK(c, cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
    if (flag) {
        CK(c, cudaMemset(c->d_err, 0, sizeof(int)), "error flag");
        return fail(c, DAFMM_ERR_TIMEOUT, "a bounded device wait gave up (site " + std::to_string(flag) + ")");
    }
#if defined(DAFMM_CHECK)
    long long index = 0, bound = 0;
    if (const int site = check_take_all(&index, &bound))
        return fail(c, DAFMM_ERR_CHECK, std::string(check_site_name(site)) + " (site " + std::to_string(site) +
                                            "): index " + std::to_string(index) + ", bound " + std::to_string(bound));
#endif
    return DAFMM_OK;
}

int dafmm_graph_create(dafmm_tree* t, int order, int precision, double* phi, double* field, void* stream,
                       dafmm_graph** out) {
    if (!t || !out) return DAFMM_ERR_INVALID_ARG;
    *out = nullptr;
    dafmm_ctx* c = t->ctx;
    if ((phi && !is_device_ptr(phi)) || (field && !is_device_ptr(field)))
        return fail(c, DAFMM_ERR_INVALID_ARG, "graph outputs must be device memory");
    CK(c, cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    // one ordinary evaluation first: every table, expansion and scratch array gets allocated
    int rc = dafmm_eval(t, order, 1.0, precision, phi, field, stream);
    if (rc) return rc;
    CK(c, cudaStreamSynchronize(s), "graph warm-up");
    if ((rc = tree_ready(t, s))) return rc;  // (the build has completed: no wait is captured)
    cudaStream_t cs = s;
    if (!cs) CK(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    const bool prof = c->profile;
    c->profile = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = dafmm_eval(t, order, 1.0, precision, phi, field, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    c->profile = prof;
    if (!s) cudaStreamDestroy(cs);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : cuda_fail(c, e, "graph capture");
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, e, "graph instantiate");
    }
    size_t nodes = 0;
    cudaGraphGetNodes(g, nullptr, &nodes);
    dafmm_graph* gr = new dafmm_graph();
    gr->ctx = c;
    gr->tree = t;
    gr->graph = g;
    gr->exec = x;
    gr->nodes = (int)nodes;
    *out = gr;
    return DAFMM_OK;
}

int dafmm_graph_launch(dafmm_graph* g, void* stream) {
    if (!g) return DAFMM_ERR_INVALID_ARG;
    CK(g->ctx, cudaSetDevice(g->ctx->device), "cudaSetDevice");
    CK(g->ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream), "graph launch");
    return DAFMM_OK;
}

int dafmm_graph_nodes(const dafmm_graph* g) { return g ? g->nodes : DAFMM_ERR_INVALID_ARG; }

int dafmm_graph_free(dafmm_graph* g) {
    if (!g) return DAFMM_ERR_INVALID_ARG;
    cudaSetDevice(g->ctx->device);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return DAFMM_OK;
}

int64_t dafmm_debug_level(const dafmm_tree* t, int which, int level, double* out, int64_t cap) {
    if (!t || !out || which < 0 || which > 5) return DAFMM_ERR_INVALID_ARG;
    const Expansions& e = t->ex;
    if (e.p < 0 || level < 2 || level > e.depth) return DAFMM_ERR_INVALID_ARG;
    const int64_t cnt = (int64_t)level_boxes(level) * ncp_of(e.p);
    if (cap < cnt) return DAFMM_ERR_INVALID_ARG;
    if (cudaSetDevice(t->ctx->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return DAFMM_ERR_CUDA;
    if ((which == 1 && e.L_f32) || (which == 0 && e.M_f32)) {
        std::vector<float> tmp(cnt);
        if (cudaMemcpy(tmp.data(), which == 0 ? (const void*)e.M[level] : (const void*)e.L[level], cnt * sizeof(float),
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return DAFMM_ERR_CUDA;
        for (int64_t i = 0; i < cnt; ++i) out[i] = tmp[i];
    } else if (which <= 1) {
        const double* src = which == 0 ? e.M[level] : e.L[level];
        if (cudaMemcpy(out, src, cnt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return DAFMM_ERR_CUDA;
    } else {
        const float* src = which == 2 ? e.Mhi[level] : which == 3 ? e.Mlo[level] : which == 4 ? e.Lhi[level] : e.Llo[level];
        std::vector<float> tmp(cnt);
        if (cudaMemcpy(tmp.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return DAFMM_ERR_CUDA;
        for (int64_t i = 0; i < cnt; ++i) out[i] = tmp[i];
    }
    if (which == 0 && e.M_harm) {
        // harmonic-basis multipoles: the device wrote the free coefficients only; the others
        // follow by Laplace's equation (in order of increasing z exponent), in FP64
        std::vector<int4> step;
        std::vector<double2> w;
        int cst[kMaxOrder + 3];
        harm_steps(e.p, step, w, cst);
        const int ncp = ncp_of(e.p), nc = ncoef_of(e.p);
        for (int64_t r = 0; r < cnt / ncp; ++r) {
            double* row = out + r * ncp;
            for (size_t q = 0; q < step.size(); ++q) row[step[q].x] = w[q].x * row[step[q].y] + w[q].y * row[step[q].z];
            for (int k = nc; k < ncp; ++k) row[k] = 0.0;
        }
    }
    return cnt;
}

int dafmm_set_profiling(dafmm_ctx* c, int enable) {
    if (!c) return DAFMM_ERR_INVALID_ARG;
    CK(c, cudaSetDevice(c->device), "cudaSetDevice");
    if (enable && !c->ev[0])
        for (int k = 0; k < 8; ++k) CK(c, cudaEventCreate(&c->ev[k]), "cudaEventCreate");
    c->profile = enable != 0;
    c->have_profile = false;
    return DAFMM_OK;
}

int dafmm_last_phase_ms(dafmm_ctx* c, double* out) {
    if (!c || !out) return DAFMM_ERR_INVALID_ARG;
    if (!c->have_profile) return fail(c, DAFMM_ERR_INVALID_ARG, "no profiled evaluation recorded");
    CK(c, cudaEventSynchronize(c->ev[7]), "event sync");
    float ms[7];
    const int a[7] = {0, 1, 3, 4, 5, 6, 2}, b[7] = {1, 2, 5, 5, 6, 7, 3};
    for (int k = 0; k < 7; ++k) CK(c, cudaEventElapsedTime(&ms[k], c->ev[a[k]], c->ev[b[k]]), "elapsed");
    float tot;
    CK(c, cudaEventElapsedTime(&tot, c->ev[0], c->ev[7]), "elapsed");
    out[0] = ms[0];  // P2M
    out[1] = ms[1];  // M2M
    out[2] = ms[2];  // M2L, all levels
    out[3] = ms[3];  // M2L, finest level
    out[4] = ms[4];  // L2L
    out[5] = ms[5];  // L2P + P2P
    out[6] = ms[6];  // conversions
    out[7] = tot;
    out[8] = c->last_launches;
    out[9] = 0.0;
    return DAFMM_OK;
}

size_t dafmm_footprint(int64_t n, int order, int uniform_depth, int max_leaf, int precision) {
    (void)precision;
    if (order < 0 || order > kMaxOrder || n < 0) return 0;
    const int depth = uniform_depth < 0 ? 0 : uniform_depth;
    size_t b = tree_bytes(n, depth);
    const size_t ncp = ncp_of(order), nc = ncoef_of(order);
    if (uniform_depth < 0) {
        // adaptive: about 16 n / max_leaf boxes; per box its hierarchy record, list entries
        // (U, W and X, about 64 on average), its first FP32 record, a padding record (with its
        // remainder record) and the expansions
        const size_t nbox = 2 + (size_t)(16 * n) / (size_t)(max_leaf > 0 ? max_leaf : 1);
        b += nbox * (kBoxInts * 4 + 64 * 4 + 24 + 32 + ncp * (8 + 8 + 4));
        b += (size_t)kNumKeys * nc * ncp * 12;
        b += (size_t)n * 12 + radix_sort_temp_bytes(n) + radix_sort_temp_bytes((int64_t)nbox);
        return b;
    }
    for (int l = 2; l <= depth; ++l) b += level_boxes(l) * ncp * (8 + 8 + 4);
    b += (size_t)kNumKeys * nc * ncp * 12;
    b += (size_t)n * 12 + radix_sort_temp_bytes(n);  // build-time scratch
    // the staging of host input arrays (xyz and q): a pooled context's asynchronous build holds
    // it, with the scratch above, until the build has completed
    b += (size_t)n * 32;
    return b;
}

// ---- single-operator batches -------------------------------------------------------------------
static int op_common(dafmm_ctx* c, int order, int precision) {
    if (!c) return DAFMM_ERR_INVALID_ARG;
    if (order < 0 || order > kMaxOrder) return fail(c, DAFMM_ERR_UNSUPPORTED_ORDER, std::to_string(order));
    if (precision != DAFMM_FP64 && precision != DAFMM_FP32 && precision != (DAFMM_FP64 | DAFMM_OP_NUMERICAL_DA))
        return fail(c, DAFMM_ERR_INVALID_ARG, "precision");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, DAFMM_ERR_CUDA, "cudaSetDevice");
    return DAFMM_OK;
}

// the numerical-DA form of an operator batch (da_numeric.cu): the order's product table, then
// one launch
static cudaError_t numerical_da(dafmm_ctx* c, int order, int op, int64_t count, const double* a, const double* b,
                                const int* oct, double* out, cudaStream_t s) {
    if (ensure_order(c, order, s, false)) return cudaErrorMemoryAllocation;
    return launch_da_op(c->ord[order], op, count, a, b, oct, out, c->num_sms, s);
}

static int finish_out(dafmm_ctx* c, double* user, void* dev, size_t bytes, bool owned, cudaStream_t s) {
    if (owned) {
        CK(c, cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, s), "D2H");
        CK(c, cudaStreamSynchronize(s), "sync");
    }
    return DAFMM_OK;
}

typedef cudaError_t (*op2_fn)(int, int64_t, const double*, const double*, double*, cudaStream_t);

static int run_op2(dafmm_ctx* c, int order, int prec, int64_t count, const double* a, size_t abytes,
                   const double* b, size_t bbytes, double* out, size_t obytes, op2_fn fn, void* stream,
                   const char* what, int da_op) {
    int rc = op_common(c, order, prec);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!a || !b || !out))) return fail(c, DAFMM_ERR_INVALID_ARG, what);
    cudaStream_t s = (cudaStream_t)stream;
    Staged sa, sb, so;
    if ((rc = stage_in(c, a, abytes, s, sa))) return rc;
    if ((rc = stage_in(c, b, bbytes, s, sb))) return rc;
    so.c = c;
    so.bytes = obytes;
    if (is_device_ptr(out) || obytes == 0) {
        so.dev = out;
    } else {
        if ((rc = dev_alloc(c, &so.dev, obytes, "op output"))) return rc;
        so.owned = true;
    }
    if (prec & DAFMM_OP_NUMERICAL_DA) {
        CK(c, numerical_da(c, order, da_op, count, (const double*)sa.dev, (const double*)sb.dev, nullptr,
                           (double*)so.dev, s),
           what);
    } else {
        CK(c, fn(prec, count, (const double*)sa.dev, (const double*)sb.dev, (double*)so.dev, s), what);
    }
    return finish_out(c, out, so.dev, obytes, so.owned, s);
}

int dafmm_op_p2m(dafmm_ctx* c, int order, int precision, int64_t count, const double* s3, const double* q,
                 double* out, void* stream) {
    const size_t nc = ncoef_of(order < 0 || order > kMaxOrder ? 0 : order);
    const OrderOps* ops = order_ops(order);
    if (!ops) return op_common(c, order, precision);
    return run_op2(c, order, precision, count, s3, count * 3 * 8, q, count * 8, out, count * nc * 8, ops->op_p2m,
                   stream, "P2M", kDaP2M);
}

int dafmm_op_p2l(dafmm_ctx* c, int order, int precision, int64_t count, const double* w, const double* q,
                 double* out, void* stream) {
    const size_t nc = ncoef_of(order < 0 || order > kMaxOrder ? 0 : order);
    const OrderOps* ops = order_ops(order);
    if (!ops) return op_common(c, order, precision);
    return run_op2(c, order, precision, count, w, count * 3 * 8, q, count * 8, out, count * nc * 8, ops->op_p2l,
                   stream, "P2L", kDaP2L);
}

int dafmm_op_l2p(dafmm_ctx* c, int order, int precision, int64_t count, const double* L, const double* x,
                 double* out4, void* stream) {
    const size_t nc = ncoef_of(order < 0 || order > kMaxOrder ? 0 : order);
    const OrderOps* ops = order_ops(order);
    if (!ops) return op_common(c, order, precision);
    return run_op2(c, order, precision, count, L, count * nc * 8, x, count * 3 * 8, out4, count * 4 * 8,
                   ops->op_l2p, stream, "L2P", kDaL2P);
}

int dafmm_op_m2p(dafmm_ctx* c, int order, int precision, int64_t count, const double* M, const double* s3,
                 double* out4, void* stream) {
    const size_t nc = ncoef_of(order < 0 || order > kMaxOrder ? 0 : order);
    const OrderOps* ops = order_ops(order);
    if (!ops) return op_common(c, order, precision);
    return run_op2(c, order, precision, count, M, count * nc * 8, s3, count * 3 * 8, out4, count * 4 * 8,
                   ops->op_m2p, stream, "M2P", kDaM2P);
}

static int run_shift(dafmm_ctx* c, int which, int order, int prec, int64_t count, const int* oct,
                     const double* in, double* out, void* stream) {
    int rc = op_common(c, order, prec);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!oct || !in || !out))) return fail(c, DAFMM_ERR_INVALID_ARG, "shift op");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_order(c, order, s, false))) return rc;
    const size_t nc = ncoef_of(order);
    Staged so_, si, sout;
    if ((rc = stage_in(c, oct, count * sizeof(int), s, so_))) return rc;
    if ((rc = stage_in(c, in, count * nc * 8, s, si))) return rc;
    sout.c = c;
    sout.bytes = count * nc * 8;
    if (is_device_ptr(out) || count == 0) {
        sout.dev = out;
    } else {
        if ((rc = dev_alloc(c, &sout.dev, sout.bytes, "op output"))) return rc;
        sout.owned = true;
    }
    if (prec & DAFMM_OP_NUMERICAL_DA) {
        CK(c, numerical_da(c, order, which == 0 ? kDaM2M : kDaL2L, count, (const double*)si.dev, nullptr,
                           (const int*)so_.dev, (double*)sout.dev, s),
           which == 0 ? "M2M" : "L2L");
    } else {
        CK(c, order_ops(order)->op_shift(c->ord[order], which, prec, count, (const int*)so_.dev,
                                         (const double*)si.dev, (double*)sout.dev, s),
           which == 0 ? "M2M" : "L2L");
    }
    return finish_out(c, out, sout.dev, sout.bytes, sout.owned, s);
}

int dafmm_op_m2m(dafmm_ctx* c, int order, int precision, int64_t count, const int* oct, const double* in,
                 double* out, void* stream) {
    return run_shift(c, 0, order, precision, count, oct, in, out, stream);
}

int dafmm_op_l2l(dafmm_ctx* c, int order, int precision, int64_t count, const int* oct, const double* in,
                 double* out, void* stream) {
    return run_shift(c, 1, order, precision, count, oct, in, out, stream);
}

int dafmm_op_m2l(dafmm_ctx* c, int order, int precision, int64_t count, const double* r0, const double* M,
                 double* out, void* stream) {
    int rc = op_common(c, order, precision);
    if (rc) return rc;
    if (!(precision & DAFMM_OP_NUMERICAL_DA))
        return fail(c, DAFMM_ERR_UNSUPPORTED, "dafmm_op_m2l: numerical DA only (DAFMM_FP64 | DAFMM_OP_NUMERICAL_DA)");
    const size_t nc = ncoef_of(order);
    return run_op2(c, order, precision, count, M, count * nc * 8, r0, count * 3 * 8, out, count * nc * 8, nullptr,
                   stream, "M2L", kDaM2L);
}

int dafmm_op_m2l_matrix(dafmm_ctx* c, int order, const int* v3, double* K, void* stream) {
    int rc = op_common(c, order, DAFMM_FP64);
    if (rc) return rc;
    if (!v3 || !K) return fail(c, DAFMM_ERR_INVALID_ARG, "M2L matrix");
    const int m = std::max(abs(v3[0]), std::max(abs(v3[1]), abs(v3[2])));
    if (m < 2 || m > 3) return fail(c, DAFMM_ERR_INVALID_ARG, "displacement must have max |v_k| in 2..3");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_order(c, order, s, true))) return rc;
    const OrderData& od = c->ord[order];
    const int key = (v3[0] + 3) * 49 + (v3[1] + 3) * 7 + (v3[2] + 3);
    std::vector<double> buf((size_t)od.nc * od.ncp);
    CK(c, cudaMemcpyAsync(buf.data(), od.K64 + (size_t)key * od.nc * od.ncp, buf.size() * 8, cudaMemcpyDeviceToHost, s),
       "K copy");
    CK(c, cudaStreamSynchronize(s), "sync");
    std::vector<double> outv((size_t)od.nc * od.nc);
    for (int b = 0; b < od.nc; ++b)
        for (int a = 0; a < od.nc; ++a) outv[(size_t)b * od.nc + a] = buf[(size_t)b * od.ncp + a];
    if (is_device_ptr(K)) {
        CK(c, cudaMemcpyAsync(K, outv.data(), outv.size() * 8, cudaMemcpyHostToDevice, s), "K copy");
        CK(c, cudaStreamSynchronize(s), "sync");
    } else {
        memcpy(K, outv.data(), outv.size() * 8);
    }
    return DAFMM_OK;
}

}  // extern "C"
