// check.cuh -- index checks of the checked build (compiled with -DDAFMM_CHECK; the paper has
// no counterpart: it is this library's stand-in for a device memory checker).
//
// The checks guard the device accesses whose index is read from memory rather than computed
// from the launch geometry: particle ranges of leaves and boxes, box indices taken from the
// tree arrays and interaction lists, list pointers, rotation task entries, sort and gather
// positions, and the source rows the gathered M2L fetches.  A failing check records (site,
// index, bound) in the translation unit's record -- the first failure wins, by compare-and-swap
// on the site word -- and the caller skips the access (an empty range, a missing box); there
// is no trap, so the context stays usable.  dafmm_sync reads and clears every translation
// unit's record and returns DAFMM_ERR_CHECK naming the first site it finds.
//
// Without DAFMM_CHECK every check is the constant `true` and the kernels compile as if the
// checks were not there.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dafmm {

enum CheckSite : int {
    kChkLeafRange = 1,     // particle range [leaf_start[l], leaf_start[l + 1]) of a uniform leaf
    kChkBoxIndex = 2,      // a box index read from an adaptive tree array or list
    kChkBoxRange = 3,      // particle range [pbeg, pend) of an adaptive box
    kChkListPtr = 4,       // a CSR list range (U, W, X lists; M2L target groups)
    kChkRotTask = 5,       // a rotation task entry (coefficient index or table offset)
    kChkRecord = 6,        // FP32 records of a leaf (its first record and count)
    kChkSortScatter = 7,   // destination of the radix sort's scatter
    kChkPerm = 8,          // an input index read from the sort permutation
    kChkLeafKey = 9,       // the leaf a sorted key falls in
    kChkSplitChild = 10,   // a child box created by the adaptive split
    kChkListFill = 11,     // a write position of the interaction-list fill
    kChkGatherSource = 12, // a source row of the gathered tensor-core M2L
    kChkDebug = 99,        // dafmm_debug_check's deliberate failure
};

// host: the name of a site code ("unknown" for others)
const char* check_site_name(int site);

#if defined(DAFMM_CHECK)
// the record of one translation unit: read and clear it (returns the site, 0 when clear)
using CheckTake = int (*)(long long* index, long long* bound);
// host: add a translation unit's reader to the list dafmm_sync walks (called at load time)
void check_register(CheckTake take);
// host: walk the list; the first site found (0 if none), each record cleared
int check_take_all(long long* index, long long* bound);

#endif

}  // namespace dafmm

#if defined(DAFMM_CHECK)
// the record of this translation unit (static: one per translation unit) and its reader
static __device__ unsigned long long dafmm_check_rec[3];  // site, index, bound of the first failure

static __device__ __noinline__ void dafmm_check_record(long long i, long long n, int site) {
    if (atomicCAS(&dafmm_check_rec[0], 0ull, (unsigned long long)site) == 0ull) {
        dafmm_check_rec[1] = (unsigned long long)i;
        dafmm_check_rec[2] = (unsigned long long)n;
    }
}

static int dafmm_check_take_tu(long long* index, long long* bound) {
    unsigned long long r[3] = {0, 0, 0};
    if (cudaMemcpyFromSymbol(r, dafmm_check_rec, sizeof(r)) != cudaSuccess) return 0;
    if (r[0] == 0) return 0;
    const unsigned long long z[3] = {0, 0, 0};
    cudaMemcpyToSymbol(dafmm_check_rec, z, sizeof(z));
    *index = (long long)r[1];
    *bound = (long long)r[2];
    return (int)r[0];
}

struct DafmmCheckRegistrar {
    explicit DafmmCheckRegistrar(dafmm::CheckTake take) { dafmm::check_register(take); }
};
static DafmmCheckRegistrar dafmm_check_registrar(&dafmm_check_take_tu);

// i in [0, n)
static __device__ __forceinline__ bool dafmm_chk_in(long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    dafmm_check_record(i, n, site);
    return false;
}
// 0 <= a <= b <= n
static __device__ __forceinline__ bool dafmm_chk_range(long long a, long long b, long long n, int site) {
    if (a >= 0 && a <= b && b <= n) return true;
    dafmm_check_record(a < 0 || a > b ? a : b, n, site);
    return false;
}
#endif

// The checks as the kernels write them: without DAFMM_CHECK they are `true` and their
// arguments are not evaluated (the bounds they name exist only in checked builds).
#if defined(DAFMM_CHECK)
#define DAFMM_IN(i, n, site) ::dafmm_chk_in((long long)(i), (long long)(n), (site))
#define DAFMM_RANGE(a, b, n, site) ::dafmm_chk_range((long long)(a), (long long)(b), (long long)(n), (site))
#else
#define DAFMM_IN(i, n, site) true
#define DAFMM_RANGE(a, b, n, site) true
#endif
