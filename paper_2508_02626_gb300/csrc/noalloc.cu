// noalloc.cu -- dafmm_eval_noalloc: an FP64 evaluation of an existing tree that allocates
// no device memory.
//
// Who needs it: callers that cannot call cudaMalloc at evaluation time -- for example a
// service that has handed all device memory to its own pool allocator, or a latency-
// critical loop where the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable.  dafmm_eval allocates its expansion arrays and operator tables on first use;
// this entry point keeps them instead in one fixed array in device memory that is part of
// the library's module (kNoAllocBytes = 32 MiB, held by every GPU that loads the library
// until the process exits).  It supports expansion orders up to 6 and uniform trees up to
// depth 4, and rejects anything larger.
//
// Set-up: the first call on a device looks up the device address of the array
// (cudaGetSymbolAddress, with that device current) and caches it.  The operator tables it
// copies in come from host storage kept for the process.  Every call shares the array and
// rewrites everything it uses, so calls that overlap on the GPU (different streams, or other
// host threads) race and must be ordered by the caller.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "api_types.h"
#include "da_common.cuh"
#include "internal.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;
constexpr int kNoAllocMaxOrder = 6;
constexpr int kNoAllocMaxDepth = 4;
constexpr int kMaxDevices = 64;

}  // namespace

// the scratch array: one copy per device that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// device address of the scratch array on `device` (which must be current); looked up once
cudaError_t scratch_address(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// carves 256-byte aligned pieces off the scratch array, in order
struct Carver {
    unsigned char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += (count * sizeof(T) + 255) / 256 * 256;
        return p;
    }
};

int set_err(dafmm_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

bool device_or_null(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host-side tables of one order that the evaluation copies into the scratch array: the DA
// product table of the K generation (pairs (i, j) with e_i + e_j = e_k per output k, and the
// index of e_k minus one unit per axis) and the per-octant row starts of the M2M/L2L tables.
// Built once per order on first use and kept until the process exits, so that every copy
// reads host memory that outlives the call that issued it.
struct HostTables {
    std::vector<int> rowptr;
    std::vector<ushort2> pairs;
    std::vector<short> minus;
    std::vector<int> m2m_rp8, l2l_rp8;
};

HostTables g_tables[kNoAllocMaxOrder + 1];
std::once_flag g_tables_once[kNoAllocMaxOrder + 1];

const HostTables& host_tables(int order) {
    std::call_once(g_tables_once[order], [order] {
        const dafmm::OrderOps* ops = dafmm::order_ops(order);
        const int nc = ops->nc;
        HostTables& ht = g_tables[order];
        std::vector<int> ex(3 * nc);
        for (int n = 0; n <= order; ++n)
            for (int a = n; a >= 0; --a)
                for (int b = n - a; b >= 0; --b) {
                    const int cc = n - a - b, k = dafmm::da_index(a, b, cc);
                    ex[3 * k] = a; ex[3 * k + 1] = b; ex[3 * k + 2] = cc;
                }
        ht.rowptr.resize(nc + 1);
        for (int k = 0; k < nc; ++k) {
            ht.rowptr[k] = (int)ht.pairs.size();
            for (int i = 0; i < nc; ++i) {
                const int r0 = ex[3 * k] - ex[3 * i], r1 = ex[3 * k + 1] - ex[3 * i + 1], r2 = ex[3 * k + 2] - ex[3 * i + 2];
                if (r0 < 0 || r1 < 0 || r2 < 0) continue;
                ushort2 pr;
                pr.x = (unsigned short)i;
                pr.y = (unsigned short)dafmm::da_index(r0, r1, r2);
                ht.pairs.push_back(pr);
            }
        }
        ht.rowptr[nc] = (int)ht.pairs.size();
        ht.minus.resize(3 * nc);
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < nc; ++k) {
                int e[3] = {ex[3 * k], ex[3 * k + 1], ex[3 * k + 2]};
                if (e[d] == 0) {
                    ht.minus[d * nc + k] = -1;
                } else {
                    e[d] -= 1;
                    ht.minus[d * nc + k] = (short)dafmm::da_index(e[0], e[1], e[2]);
                }
            }
        ht.m2m_rp8.resize(8 * (size_t)nc + 1);
        ht.l2l_rp8.resize(8 * (size_t)nc + 1);
        dafmm::shift_rp8(ops->m2m, nc, ht.m2m_rp8.data());
        dafmm::shift_rp8(ops->l2l, nc, ht.l2l_rp8.data());
    });
    return g_tables[order];
}

}  // namespace

using namespace dafmm;

extern "C" int dafmm_eval_noalloc(dafmm_tree* t, int order, double* phi, double* field, void* stream) {
    if (!t) return DAFMM_ERR_INVALID_ARG;
    dafmm_ctx* c = t->ctx;
    if (order < 0 || order > kNoAllocMaxOrder)
        return set_err(c, DAFMM_ERR_UNSUPPORTED_ORDER,
                       "dafmm_eval_noalloc: order " + std::to_string(order) + " above its limit of 6");
    if (t->adaptive)
        return set_err(c, DAFMM_ERR_UNSUPPORTED, "dafmm_eval_noalloc: uniform trees only");
    if (t->depth > kNoAllocMaxDepth)
        return set_err(c, DAFMM_ERR_INVALID_ARG,
                       "dafmm_eval_noalloc: tree depth " + std::to_string(t->depth) + " above its limit of 4");
    if (c->device < 0 || c->device >= kMaxDevices) return set_err(c, DAFMM_ERR_INVALID_ARG, "device index");
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, DAFMM_ERR_CUDA, "cudaSetDevice");
    if (!device_or_null(phi) || !device_or_null(field))
        return set_err(c, DAFMM_ERR_INVALID_ARG, "dafmm_eval_noalloc: outputs must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    if (tree_ready(t, s) != DAFMM_OK) return set_err(c, DAFMM_ERR_CUDA, "dafmm_eval_noalloc: tree build");
    if (t->n == 0) return DAFMM_OK;
    const OrderOps* ops = order_ops(order);
    const int nc = ops->nc, ncp = ops->ncp;
    const bool far = t->depth >= 2;

    const HostTables& ht = host_tables(order);
    const std::vector<int>& rowptr = ht.rowptr;
    const std::vector<ushort2>& pairs = ht.pairs;
    const std::vector<short>& minus = ht.minus;

    // plan the layout (a dry run with a null base gives the size)
    auto plan = [&](unsigned char* base, OrderData& od, double** M, double** L) {
        Carver cv{base};
        od.p = order;
        od.nc = nc;
        od.ncp = ncp;
        od.m2m_rowptr = cv.take<int>(nc + 1);
        od.m2m_col = cv.take<unsigned short>(ops->m2m.nnz);
        od.m2m_par = cv.take<unsigned char>(ops->m2m.nnz);
        od.m2m_val = cv.take<double>(ops->m2m.nnz);
        od.l2l_rowptr = cv.take<int>(nc + 1);
        od.l2l_col = cv.take<unsigned short>(ops->l2l.nnz);
        od.l2l_par = cv.take<unsigned char>(ops->l2l.nnz);
        od.l2l_val = cv.take<double>(ops->l2l.nnz);
        od.m2m_rp8 = cv.take<int>(8 * (size_t)nc + 1);
        od.l2l_rp8 = cv.take<int>(8 * (size_t)nc + 1);
        od.mul_rowptr = cv.take<int>(rowptr.size());
        od.mul_pairs = cv.take<ushort2>(pairs.size());
        od.mul_minus = cv.take<short>(minus.size());
        od.K64 = far ? cv.take<double>((size_t)kNumKeys * nc * ncp) : nullptr;
        for (int l = 2; l <= t->depth; ++l) {
            const size_t cnt = ((size_t)1 << (3 * l)) * ncp;
            M[l] = cv.take<double>(cnt);
            L[l] = cv.take<double>(cnt);
        }
        return cv.off;
    };
    OrderData od;
    double* M[kMaxUniformDepth + 1] = {};
    double* L[kMaxUniformDepth + 1] = {};
    const size_t need = plan(nullptr, od, M, L);
    if (need > kNoAllocBytes)
        return set_err(c, DAFMM_ERR_INVALID_ARG,
                       "dafmm_eval_noalloc: needs " + std::to_string(need) + " bytes of scratch, above its " +
                           std::to_string(kNoAllocBytes) + "-byte array");
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(c->device, &base);
    if (e != cudaSuccess) return set_err(c, DAFMM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    od = OrderData();
    plan(base, od, M, L);

    // operator tables into the scratch array (no reliance on what an earlier call left there)
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    up(od.m2m_rowptr, ops->m2m.rowptr, (nc + 1) * sizeof(int));
    up(od.m2m_col, ops->m2m.col, ops->m2m.nnz * sizeof(unsigned short));
    up(od.m2m_par, ops->m2m.par, ops->m2m.nnz);
    up(od.m2m_val, ops->m2m.val, ops->m2m.nnz * sizeof(double));
    up(od.l2l_rowptr, ops->l2l.rowptr, (nc + 1) * sizeof(int));
    up(od.l2l_col, ops->l2l.col, ops->l2l.nnz * sizeof(unsigned short));
    up(od.l2l_par, ops->l2l.par, ops->l2l.nnz);
    up(od.l2l_val, ops->l2l.val, ops->l2l.nnz * sizeof(double));
    up(od.m2m_rp8, ht.m2m_rp8.data(), ht.m2m_rp8.size() * sizeof(int));
    up(od.l2l_rp8, ht.l2l_rp8.data(), ht.l2l_rp8.size() * sizeof(int));
    up(od.mul_rowptr, rowptr.data(), rowptr.size() * sizeof(int));
    up(od.mul_pairs, pairs.data(), pairs.size() * sizeof(ushort2));
    up(od.mul_minus, minus.data(), minus.size() * sizeof(short));
    for (int l = 2; l <= t->depth && e == cudaSuccess; ++l) {
        const size_t cnt = ((size_t)1 << (3 * l)) * ncp;
        e = cudaMemsetAsync(M[l], 0, cnt * sizeof(double), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L[l], 0, cnt * sizeof(double), s);
    }
    if (e != cudaSuccess) return set_err(c, DAFMM_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));

    // the FP64 evaluation sequence of dafmm_eval, on the scratch buffers
    const TreeView tv = make_view(t);
    const int Ld = t->depth;
    if (far) {
        if (e == cudaSuccess) e = ops->kgen(od, nullptr, kNumKeys, s);
        if (e == cudaSuccess) e = ops->p2m(tv, DAFMM_FP64, M[Ld], nullptr, s);
        for (int lc = Ld; lc >= 3 && e == cudaSuccess; --lc) e = ops->m2m_level(od, DAFMM_FP64, lc, M[lc], M[lc - 1], s);
        for (int l = 2; l <= Ld && e == cudaSuccess; ++l)
            e = ops->m2l_level(od, DAFMM_FP64, l, M[l], nullptr, L[l], 1.0 / ldexp(t->dom[3], -l), s);
        for (int lc = 3; lc <= Ld && e == cudaSuccess; ++lc) e = ops->l2l_level(od, DAFMM_FP64, lc, L[lc - 1], L[lc], s);
    }
    if (e == cudaSuccess) e = ops->leaf(tv, DAFMM_FP64, far ? L[Ld] : nullptr, phi, field, s);
    if (e != cudaSuccess) return set_err(c, DAFMM_ERR_CUDA, std::string("dafmm_eval_noalloc: ") + cudaGetErrorString(e));
    return DAFMM_OK;
}
