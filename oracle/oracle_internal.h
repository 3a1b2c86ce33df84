/* oracle_internal.h -- shared declarations between the oracle's own C files.
 * TEST INFRASTRUCTURE ONLY (see oracle.h). */
#ifndef DAFMM_ORACLE_INTERNAL_H
#define DAFMM_ORACLE_INTERNAL_H
#include <stdint.h>
#include "oracle.h"

#define TPSA_MAXCOEF ((OR_MAXORD + 1) * (OR_MAXORD + 2) * (OR_MAXORD + 3) / 6)

typedef struct {
    int order, ncoef;
    int (*e)[3];    /* exponents of each coefficient */
    int* ord;       /* total order of each coefficient */
    int nmul;       /* entries of the product table */
    int (*mul)[3];  /* (i, j, k): a_i b_j contributes to c_k */
    int* row;       /* mul entries of left index i are row[i] .. row[i+1]-1 */
} tpsa_ctx;

int tpsa_index(int a, int b, int c);
const tpsa_ctx* tpsa_get(int order);
void da_zero(const tpsa_ctx* t, double* a);
void da_const(const tpsa_ctx* t, double* a, double c);
void da_copy(const tpsa_ctx* t, const double* a, double* c);
void da_axpy(const tpsa_ctx* t, double s, const double* a, double* c);
void da_mul(const tpsa_ctx* t, const double* a, const double* b, double* c);
int  da_pow(const tpsa_ctx* t, const double* a, double s, double* c);
void da_deriv(const tpsa_ctx* t, const double* a, int v, double* c);
double da_eval(const tpsa_ctx* t, const double* a, const double* x);
void da_monomials(const tpsa_ctx* tf, const tpsa_ctx* tg, const double* const g[3], double* mono);
void da_compose(const tpsa_ctx* tf, const double* f, const tpsa_ctx* tg, const double* const g[3],
                double* out);

/* the operators on one instance (ops.c) */
void op_p2m1(const tpsa_ctx* t, const double* s, double q, double* M);
void op_m2m(const tpsa_ctx* t, const double* M, const double* r0, double* out);
void op_m2l_map(const tpsa_ctx* t, const double* r0, double* sqrtR, double* map3);
void op_m2l(const tpsa_ctx* t, const double* M, const double* r0, double* out);
void op_m2l_rot(const tpsa_ctx* t, const double* M, const double* r0, double* out);
void op_rotation(const double* r0, double* Q);
void op_linmap(const tpsa_ctx* t, const double* a, const double* A, double* out);
void op_p2l1(const tpsa_ctx* t, const double* w, double q, double* L);
void op_l2l(const tpsa_ctx* t, const double* L, const double* r0, double* out);
void op_l2p1(const tpsa_ctx* t, const double* L, const double* x, double* phi, double* grad);
void op_m2p1(const tpsa_ctx* t, const double* M, const double* s, double* phi, double* grad);

/* a minimal parallel-for over [0, n) with pthreads */
typedef void (*pfor_fn)(int64_t begin, int64_t end, void* arg);
void parallel_for(int64_t n, int nthreads, pfor_fn fn, void* arg);
#endif
