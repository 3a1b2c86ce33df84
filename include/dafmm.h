/*
 * dafmm.h -- C ABI of the GB300 (sm_103a) DA-based fast multipole method for the
 * Coulomb potential and field (arXiv 2508.02626, "Boosting the Efficiency of the
 * Differential Algebra-based Fast Multipole Method Using Symbolic Differential
 * Algebra").
 *
 * The method (paper Sec. 1-3): particles are grouped in an octree; far
 * interactions go through Taylor (DA) expansions built by seven operators --
 * P2M (Eq. 2), M2M (Eq. 4), M2L (Eq. 5), P2L (Eq. 6), L2L (Eq. 7), L2P and M2P
 * (Sec. 3.2) -- and near interactions are summed pairwise (Sec. 1).  The
 * operators run as straight-line code generated per expansion order by a
 * symbolic DA (Sec. 3); M2L is batched over every well-separated box pair
 * (at most 189 per box, Sec. 3.4) as dense contractions grouped by
 * displacement.
 *
 * Conventions for every entry point
 *   - Return value: DAFMM_OK (0) on success, a negative DAFMM_ERR_* code
 *     otherwise; nothing aborts.  dafmm_last_error() gives a message.
 *   - Pointers to particle data and outputs may be host or device memory
 *     (detected per call).  The caller owns them; the library never keeps
 *     them beyond the call, except that results are complete only once the
 *     given stream has reached the call (host outputs: on return).
 *   - Coordinates are row-major n x 3 doubles; charges n doubles.
 *   - Potential phi_i = sum_{j != i, r_ij > 0} q_j / r_ij (Eq. 1, no Coulomb
 *     constant); field E_i = -grad phi_i, n x 3 doubles, in the input order.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - The library owns trees and contexts until *_free / dafmm_destroy.
 *   - One context must not be used from two host threads at the same time.
 */
#ifndef DAFMM_H
#define DAFMM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define DAFMM_OK 0
#define DAFMM_ERR_INVALID_ARG (-1)
#define DAFMM_ERR_UNSUPPORTED_ORDER (-2) /* order outside 0..10, the generated range (Sec. 3) */
#define DAFMM_ERR_OVER_BUDGET (-3)       /* the context's HBM budget would be exceeded */
#define DAFMM_ERR_CUDA (-4)              /* a CUDA runtime call failed */
#define DAFMM_ERR_TIMEOUT (-5)           /* a bounded device wait gave up */
#define DAFMM_ERR_UNSUPPORTED (-6)       /* a valid but unimplemented option (e.g. theta != 1) */
#define DAFMM_ERR_NO_DEVICE (-7)
#define DAFMM_ERR_CANCELLED (-8)         /* a served request dropped because its server stopped */
#define DAFMM_ERR_CHECK (-9)             /* an index check of a checked build (DAFMM_CHECK) failed */

/* arithmetic of an evaluation */
#define DAFMM_FP64 0  /* every step in double precision */
#define DAFMM_MIXED 1 /* FP32 bulk (P2M, M2L, L2P, P2P); FP64 derivative tensors, M2M/L2L, final sums */
#define DAFMM_FP32 2  /* FP32 everywhere except the derivative tensors and the final sums */
#define DAFMM_FF 3    /* FP64-level accuracy with float-float (pairs of FP32 numbers, ~48 significand
                         bits) for P2M, M2L (by rotation, Sec. 3.4) and the leaves (P2P, L2P) of
                         uniform trees, FP64 for the rest; adaptive trees and forests: as DAFMM_FP64.
                         A particle's offset from its leaf centre is held to 2^-49 leaf widths, so a
                         pair closer than about 1e-3 leaf widths has its difference accurate to that
                         absolute size rather than to FP64's relative one. */

#define DAFMM_MAX_ORDER 10

typedef struct dafmm_ctx dafmm_ctx;
typedef struct dafmm_tree dafmm_tree;
typedef struct dafmm_graph dafmm_graph;
typedef struct dafmm_server dafmm_server;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device memory the
 * context may hold (0 = no cap).  *ctx receives the handle. */
int dafmm_create(dafmm_ctx** ctx, int device, size_t hbm_budget_bytes);
/* A pooled context: it reserves pool_bytes (>= 1 MiB) of device memory at once and carves
 * every later allocation out of that reservation, first fit, 256-byte aligned (the paper
 * has no counterpart; this serves long-running loops).  Returning memory to the pool never
 * synchronises the device, unlike cudaFree, so trees can be freed while other streams run;
 * a tree must not be freed before the work that uses it has completed.  Allocations beyond
 * the pool fail with DAFMM_ERR_OVER_BUDGET. */
int dafmm_create_pooled(dafmm_ctx** ctx, int device, size_t pool_bytes);
/* Release a context and every tree it owns. */
void dafmm_destroy(dafmm_ctx* ctx);
/* Message of the last failure on this context (never NULL). */
const char* dafmm_last_error(const dafmm_ctx* ctx);
/* Device bytes currently held by the context. */
size_t dafmm_bytes_in_use(const dafmm_ctx* ctx);

/* Build an octree over n particles (Sec. 1): particles are copied into device memory,
 * sorted by box, and the interaction lists are prepared.
 *   domain        {x0, y0, z0, size} of the root cube, or NULL for the smallest cube
 *                 containing every point, enlarged by 1e-12 of its size;
 *   uniform_depth >= 0: a uniform tree with 8^depth leaves (depth <= 7);
 *                 < 0: adaptive: a box with more than max_leaf (>= 1) particles is split
 *                 into its non-empty children (Sec. 3.5), down to level 20 at most; the
 *                 far field then runs over the interaction lists of Cheng, Greengard and
 *                 Rokhlin: V (M2L), U (P2P), W (M2P) and X (P2L).
 * Box membership: k = floor((x - x0) * 2^21 / size), clamped to [0, 2^21), per axis; a box
 * of level l holds the particles whose k >> (21 - l) equal its integer coordinates.
 * Ordering: the call returns once the host arrays have been copied (they may then be reused).
 * A pooled context building a uniform tree from host arrays leaves the rest of the build in
 * flight on `stream`; every later call on the tree (on any stream) is ordered after it.
 * Otherwise the call returns with the tree built. 
 * Errors: DAFMM_ERR_INVALID_ARG for n < 0, missing arrays, max_leaf < 1 on an adaptive
 * tree, depth > 7 or a bad domain; DAFMM_ERR_OVER_BUDGET when the context's budget or the
 * device runs out of memory. */
int dafmm_build_tree(dafmm_ctx* ctx, const double* xyz, const double* q, int64_t n,
                     const double* domain, int uniform_depth, int max_leaf, void* stream,
                     dafmm_tree** tree);
/* A forest: `ntrees` independent problems in one adaptive structure, so that one evaluation
 * (a fixed number of kernel launches, independent of ntrees) solves them all.  Particles of
 * problem r are [offsets[r], offsets[r+1]) of xyz/q (offsets: ntrees + 1 host int64,
 * offsets[0] = 0, non-decreasing); problem r gets its own root cube -- domains[4r..4r+3] =
 * {x0, y0, z0, size}, or, with domains NULL, the smallest cube around its points enlarged by
 * 1e-12 of its size -- and its own adaptive tree with leaves of at most max_leaf particles
 * (Sec. 3.5).  No interaction crosses problems: each problem's potential and field are those
 * of a tree built for it alone, computed by the same arithmetic in the same order.  Outputs
 * of dafmm_eval on a forest are in the concatenated input order.
 *   Errors: DAFMM_ERR_INVALID_ARG for bad offsets, arrays, max_leaf < 1 or domains;
 *   DAFMM_ERR_OVER_BUDGET when memory runs out. */
int dafmm_build_forest(dafmm_ctx* ctx, const double* xyz, const double* q, const int64_t* offsets,
                       int ntrees, const double* domains, int max_leaf, void* stream,
                       dafmm_tree** tree);
/* Number of problems in a forest (1 for a tree) and their root cubes (4 doubles each) when
 * domains is not NULL. */
int dafmm_forest_info(const dafmm_tree* tree, int* ntrees, double* domains);
int dafmm_tree_free(dafmm_tree* tree);
/* info[0..7] = n, depth (the finest level of an adaptive tree), leaves, boxes, max particles
 * per leaf, adaptive (0/1), M2L pairs (V list entries), P2P leaf pairs (U list entries).
 * Also writes the root cube to domain4 when it is not NULL. */
int dafmm_tree_info(const dafmm_tree* tree, int64_t* info8, double* domain4);

/* Evaluate potential and field of every particle with the FMM of expansion order `order`.
 *   theta      well-separation distance in box widths; 1.0 is the paper's nearest-neighbour
 *              criterion (at most 189 M2L partners per box, Sec. 3.4) and the only value
 *              supported (others return DAFMM_ERR_UNSUPPORTED);
 *   precision  DAFMM_FP64, DAFMM_MIXED or DAFMM_FP32;
 *   phi        n doubles (may be NULL), field n x 3 doubles (may be NULL), input order. */
int dafmm_eval(dafmm_tree* tree, int order, double theta, int precision, double* phi,
               double* field, void* stream);

/* CUDA-graph form of dafmm_eval (the paper has no counterpart; it removes the per-kernel
 * launch cost of repeated evaluations).  dafmm_graph_create runs one ordinary evaluation
 * (so that every table and array exists), then records a second one on `stream` (a private
 * stream when NULL) into a graph.  Launching the graph recomputes phi and field of the same
 * tree, order and precision into the same device buffers (phi, field: device memory or
 * NULL).  The graph refers to the tree's arrays: free it before the tree.  dafmm_graph_nodes: kernels and copies in the graph. */
int dafmm_graph_create(dafmm_tree* tree, int order, int precision, double* phi, double* field,
                       void* stream, dafmm_graph** graph);
int dafmm_graph_launch(dafmm_graph* graph, void* stream);
int dafmm_graph_nodes(const dafmm_graph* graph);
int dafmm_graph_free(dafmm_graph* graph);

/* ---- serving: a request loop with continuous batching (the paper has no counterpart) ----
 * dafmm_server_create starts a scheduler thread that owns a pooled context of pool_bytes on
 * `device` and `slots` CUDA streams.  Requests (one independent problem each) may be
 * submitted from any thread at any time.  Whenever a slot is free the scheduler forms a job:
 * the oldest request and, behind it in arrival order, further requests of the same order,
 * precision and leaf size -- at most max_batch requests and max_job_particles particles,
 * and only while the job's device-memory estimate (dafmm_footprint) fits the free pool.
 * A job is one forest (dafmm_build_forest) and one dafmm_eval on the slot's stream; jobs
 * on different slots overlap on the device.  Each request's result is the one a
 * stand-alone adaptive solve of it gives (its own tree), bit for bit.
 *   dafmm_server_submit: xyz (n x 3), q (n), phi (n), field (n x 3, may be NULL) stay owned
 *     by the caller and must remain valid until dafmm_server_wait returns for that request;
 *     page-locked host or device memory lets copies overlap (pageable memory works but
 *     serialises the loop).  *id receives the request's handle.
 *   dafmm_server_wait: blocks up to timeout_s seconds (< 0: no limit) for the request;
 *     returns its status (DAFMM_OK, or the error of its job; DAFMM_ERR_OVER_BUDGET when it
 *     cannot fit the empty pool; DAFMM_ERR_CANCELLED when the server stopped first) and
 *     forgets it, or DAFMM_ERR_TIMEOUT and keeps it; DAFMM_ERR_INVALID_ARG for an id it does
 *     not hold (never submitted, already waited for, or taken by another thread waiting for
 *     the same id).  times3 (may be NULL) receives, in milliseconds: submit to results in the
 *     caller's buffers, submit to admission, and admission to results.
 *   dafmm_server_last_error: the server's last failure message, copied per calling thread
 *     (valid until that thread calls it again).
 *   dafmm_server_stats: out8 = {completed, failed, queued, running jobs, jobs launched,
 *     mean requests per job, peak pool bytes in use, peak concurrent jobs}.
 *   dafmm_server_destroy: lets running jobs finish, cancels queued requests, frees all. */
int dafmm_server_create(int device, size_t pool_bytes, int slots, int max_batch,
                        int64_t max_job_particles, dafmm_server** server);
int dafmm_server_submit(dafmm_server* server, const double* xyz, const double* q, int64_t n,
                        int order, int precision, int max_leaf, double* phi, double* field,
                        int64_t* id);
int dafmm_server_wait(dafmm_server* server, int64_t id, double timeout_s, double* times3);
int dafmm_server_stats(dafmm_server* server, double* out8);
const char* dafmm_server_last_error(dafmm_server* server);
int dafmm_server_destroy(dafmm_server* server);

/* Per-phase device time of the last dafmm_eval on this context, measured with CUDA events
 * recorded on that call's stream while profiling is enabled (dafmm_set_profiling).
 * out10 = {P2M, M2M, M2L (all levels), M2L finest level, L2L, L2P+P2P, conversions,
 * total, kernel launches, 0}; times in milliseconds.  Waits for the recorded events. */
int dafmm_set_profiling(dafmm_ctx* ctx, int enable);
int dafmm_last_phase_ms(dafmm_ctx* ctx, double* out10);

/* Options of a context.
 *   DAFMM_OPT_M2L_KERNEL: 0 = tensor-core M2L (tcgen05 split products: F16 splits in the
 *   FP32 mode unless DAFMM_OPT_M2L_F16 is 0, TF32 splits in the MIXED mode) for the FP32
 *   bulk paths when the order is >= 2 (default), 1 = SIMT FP32 M2L. */
#define DAFMM_OPT_M2L_KERNEL 1
/*   DAFMM_OPT_TC_MASK: which contractions may use the tensor cores in the FP32 mode
 *   (bit 0 M2L, bit 1 M2M, bit 2 L2L; default 5: the octant-transformed SIMT M2M is the
 *   faster one); the others run on the SIMT kernels. */
#define DAFMM_OPT_TC_MASK 2
/*   DAFMM_OPT_LEAF_WARPS: leaves per thread block of the adaptive near-field kernel (P2P,
 *   M2P, L2P), one warp each: 1, 2, 4 (default) or 8 -- the P2P tile the autotuner picks. */
#define DAFMM_OPT_LEAF_WARPS 3
/*   DAFMM_OPT_M2L_F16: operands of the FP32 mode's tensor-core M2L: 1 (default) = F16 hi/lo
 *   splits with power-of-two scales per box, per matrix row and per matrix (twice the TF32
 *   rate; FP32-level error, within a few times that of a plain FP32 product), 0 = TF32 hi/lo
 *   splits.  MIXED always uses the TF32 splits. */
#define DAFMM_OPT_M2L_F16 4
/*   DAFMM_OPT_M2L_ROTATION: the FP64 M2L (Sec. 3.4): 0 = the dense K^_v
 *   matrix of each displacement; 1 = rotate the source expansion so that the displacement lies
 *   on the x axis, apply Eq. 5 along the axis (a sparse matrix per distinct length |v|), rotate
 *   back -- per well-separated pair about 6.2k instead of 27k multiply-adds at p = 8, 14.7k
 *   instead of 82k at p = 10; -1 (default) = 1 from p = 4, else 0.  Uniform and adaptive trees
 *   (the V-list pairs of a level have the same 316 box displacements). */
#define DAFMM_OPT_M2L_ROTATION 5
/*   DAFMM_OPT_M2L_HARMONIC: the tensor-core M2L of the FP32 (F16 operands) and MIXED (TF32)
 *   modes, uniform and adaptive trees and forests: 1 (default) = in the harmonic basis.  The homogeneous parts of the multipole expansions
 *   (Eq. 2: the Legendre generating function) and of the local expansions (Taylor polynomials
 *   of a harmonic potential) are harmonic polynomials, each fixed by its coefficients of z
 *   exponent <= 1; the M2L contracts those (p + 1)^2 coefficients against K^_v restricted and
 *   composed accordingly (81 instead of 165 at p = 8) and restores the others by Laplace's
 *   equation -- the same result up to rounding with about a quarter of the multiply-adds.
 *   The P2M and the M2M then compute the multipoles' free coefficients only (the M2M by its
 *   table composed with that expansion; adaptive trees fill in the rest for the M2P).
 *   0 = all ncoef coefficients. */
#define DAFMM_OPT_M2L_HARMONIC 6
int dafmm_set_option(dafmm_ctx* ctx, int option, int64_t value);

/* Diagnostics: copy level `level` of an internal expansion array of the last evaluation
 * into host memory `out` as doubles (8^level x ncp values; ncp = ncoef rounded up to 8).
 * which: 0 multipoles, 1 locals, 2/3 TF32 high/low parts of the multipoles, 4/5 of the
 * locals.  The FP32 mode keeps the locals (M2L and L2L on tensor cores) and the multipoles
 * (F16 M2L, SIMT M2M) in FP32; they are returned as doubles all the same.  With the harmonic basis
 * (DAFMM_OPT_M2L_HARMONIC, uniform trees, FP32 and MIXED) the device computes only the multipoles'
 * (p + 1)^2 free coefficients (z exponent <= 1); the others are filled in here from Laplace's
 * equation.  Synchronises the device.  Returns the number of values, or a negative code. */
int64_t dafmm_debug_level(const dafmm_tree* tree, int which, int level, double* out, int64_t cap);

/* Wait for `stream` and report failures recorded on the device by bounded waits inside the
 * kernels (DAFMM_ERR_TIMEOUT); clears the record. */
int dafmm_sync(dafmm_ctx* ctx, void* stream);
/* Self-test of that path (the paper has no counterpart): launch on `stream` one kernel whose
 * bounded mbarrier wait -- the wait the tensor-core kernels use, at most 1 s of device time --
 * waits for an arrival that never comes, gives up, records site code 90 in the context's
 * failure record and returns.  The next dafmm_sync on the context then returns
 * DAFMM_ERR_TIMEOUT (its message names the site) and clears the record; the context and its
 * trees stay usable.  Returns DAFMM_OK once the kernel is launched, DAFMM_ERR_CUDA if the
 * launch fails, DAFMM_ERR_INVALID_ARG for a NULL context. */
int dafmm_debug_expire_wait(dafmm_ctx* ctx, void* stream);
/* The checked build (the paper has no counterpart).  A library compiled with -DDAFMM_CHECK
 * guards every device access whose index is read from memory (particle ranges of leaves and
 * boxes, box indices from the tree arrays and interaction lists, list pointers, rotation task
 * entries, sort and gather positions, the gathered M2L's source rows): a failing check records
 * its site code, the index and the bound, and the access is skipped -- no trap.  dafmm_sync
 * then returns DAFMM_ERR_CHECK, its message naming the site, index and bound, and clears the
 * record; the context stays usable (the results of that evaluation are not).  The record is
 * per device, shared by the contexts on it.
 * dafmm_debug_check launches on `stream` one kernel whose check fails on purpose (site code
 * 99: index 32 against the bound 32; the guarded array holds 64 entries, so the access would be
 * in bounds even unchecked).  Returns DAFMM_OK once launched; DAFMM_ERR_UNSUPPORTED in a
 * library built without DAFMM_CHECK; DAFMM_ERR_CUDA if the launch fails;
 * DAFMM_ERR_INVALID_ARG for a NULL context. */
int dafmm_debug_check(dafmm_ctx* ctx, void* stream);

/* dafmm_eval without device allocation.  (The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc while they evaluate -- a service whose device memory
 * all belongs to its own pool allocator, or a latency-critical loop that cannot afford the
 * implicit synchronisation of cudaMalloc/cudaFree.)  Computes the same potential and field
 * as dafmm_eval(tree, order, 1.0, DAFMM_FP64, ...) with every intermediate array (operator
 * tables, M2L matrices, multipole and local expansions) in one fixed 32 MiB array of device
 * memory that belongs to the library and stays reserved on each GPU that loads it until
 * the process exits.
 *   Limits: order <= 6 (else DAFMM_ERR_UNSUPPORTED_ORDER), uniform trees of depth <= 4
 *   (else DAFMM_ERR_INVALID_ARG; adaptive trees: DAFMM_ERR_UNSUPPORTED); phi and field must
 *   be device memory or NULL.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   and keeps it.  All calls share the array: calls that overlap on the GPU
 *   (other streams, other host threads) race, so the caller must order them. */
int dafmm_eval_noalloc(dafmm_tree* tree, int order, double* phi, double* field, void* stream);

/* Unit rates of a GPU, measured (the paper has no counterpart: these are the denominators of
 * the rooflines of the kernels bound by neither HBM nor the BF16 tensor rate).  Runs one probe
 * kernel of the given kind on `device` for about 20-100 ms after one shorter warm-up launch,
 * timed with CUDA events, and returns in *rate the counted operations per second of the whole
 * GPU and in *ms (if not NULL) the timed launch's duration:
 *   DAFMM_PEAK_FFMA      FP32 FMA, 2 flops each            DAFMM_PEAK_FFMA2  packed FP32x2 FMA, 4 flops each
 *   DAFMM_PEAK_DFMA      FP64 FMA, 2 flops each            DAFMM_PEAK_RSQRT  rsqrt.approx.f32 results
 *   DAFMM_PEAK_MMA_TF32  tcgen05.mma kind::tf32 flops      DAFMM_PEAK_MMA_F16 tcgen05.mma kind::f16 flops
 * (ALU probes: 16 independent dependency chains per thread, 8 blocks of 256 threads per SM;
 * MMA probes: one CTA per SM issuing M=128 N=256 MMAs from shared memory into TMEM.)  The
 * clocks are whatever the GPU runs at: the caller records them.  Errors: DAFMM_ERR_INVALID_ARG
 * (unknown kind, NULL rate, bad device), DAFMM_ERR_CUDA (a launch or copy failed),
 * DAFMM_ERR_TIMEOUT (the MMA probe's bounded wait for its MMAs gave up). */
#define DAFMM_PEAK_FFMA 0
#define DAFMM_PEAK_FFMA2 1
#define DAFMM_PEAK_DFMA 2
#define DAFMM_PEAK_RSQRT 3
#define DAFMM_PEAK_MMA_TF32 4
#define DAFMM_PEAK_MMA_F16 5
int dafmm_probe_peak(int device, int kind, double* rate, double* ms);

/* Device bytes an evaluation of a tree with these parameters needs (an upper estimate; for a
 * uniform tree it includes the build's scratch and the staging of host input arrays, which a
 * pooled context's asynchronous build keeps until the build has completed). */
size_t dafmm_footprint(int64_t n, int order, int uniform_depth, int max_leaf, int precision);

/* ---- single-operator batches (the paper's per-operator verification, Sec. 3) --------
 * Each entry applies one generated operator to `count` independent instances, in box-
 * scaled variables (a box of width 1): multipoles M~_a = M_a / h^|a|, locals
 * L~_b = L_b h^|b|.  Arrays are device or host memory; outputs are overwritten.
 *   precision: DAFMM_FP64 or DAFMM_FP32 (arithmetic of the generated code), or
 *   DAFMM_FP64 | DAFMM_OP_NUMERICAL_DA: the same operator evaluated step by step with
 *   numerical DA (truncated power series arithmetic, Appendix A: products truncated at
 *   order p, powers by the binomial series, composition with the operator's map), FP64, one
 *   warp per instance -- the baseline the generated code replaces (Sec. 3, Tables 2-8).
 *   Any other value: DAFMM_ERR_INVALID_ARG. */
#define DAFMM_OP_NUMERICAL_DA 16

/* P2M, Eq. 2: out[i*nc + k] = q_i * coefficient k of (1 - 2 s_i.d + s_i^2 d^2)^(-1/2) */
int dafmm_op_p2m(dafmm_ctx* ctx, int order, int precision, int64_t count, const double* s,
                 const double* q, double* out, void* stream);
/* P2L, Eq. 6: out[i*nc + k] = q_i * coefficient k of 1/|w_i + d'| */
int dafmm_op_p2l(dafmm_ctx* ctx, int order, int precision, int64_t count, const double* w,
                 const double* q, double* out, void* stream);
/* L2P (Sec. 3.2): out4[i] = (L_i(x_i), grad L_i(x_i)); L is count x nc */
int dafmm_op_l2p(dafmm_ctx* ctx, int order, int precision, int64_t count, const double* L,
                 const double* x, double* out4, void* stream);
/* M2P (Sec. 3.2): out4[i] = (|d| M_i(d), grad_s), d = s_i/|s_i|^2 */
int dafmm_op_m2p(dafmm_ctx* ctx, int order, int precision, int64_t count, const double* M,
                 const double* s, double* out4, void* stream);
/* M2M, Eq. 4 (child width 1, parent width 2) and L2L, Eq. 7 (parent width 1, child width
 * 1/2) for child octant oct[i] (bit v set = upper half along axis v); in/out count x nc */
int dafmm_op_m2m(dafmm_ctx* ctx, int order, int precision, int64_t count, const int* oct,
                 const double* in, double* out, void* stream);
int dafmm_op_l2l(dafmm_ctx* ctx, int order, int precision, int64_t count, const int* oct,
                 const double* in, double* out, void* stream);
/* M2L, Eq. 5, by numerical DA only (precision must be DAFMM_FP64 | DAFMM_OP_NUMERICAL_DA, else
 * DAFMM_ERR_UNSUPPORTED; the generated M2L runs inside dafmm_eval, and its matrices come from
 * dafmm_op_m2l_matrix): out[i*nc + b] = coefficient b of sqrt(R) (M_i o M2), M2: d = (r0_i + d') R,
 * R = 1/|r0_i + d'|^2, for the displacement r0_i = r0[3i .. 3i+2] (target centre - source
 * centre, boxes of width 1; any well-separated real vector); M is count x nc. */
int dafmm_op_m2l(dafmm_ctx* ctx, int order, int precision, int64_t count, const double* r0, const double* M,
                 double* out, void* stream);
/* M2L matrix of Eq. 5 for an integer box displacement v (target - source, boxes of width 1,
 * max|v_k| in 2..3): K[b*nc + a] = coefficient b of M2L(e_a), computed on the GPU in FP64. */
int dafmm_op_m2l_matrix(dafmm_ctx* ctx, int order, const int* v3, double* K, void* stream);

#ifdef __cplusplus
}
#endif
#endif
