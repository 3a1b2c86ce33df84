/*
 * oracle.h -- CPU FP64 oracle for the DA-based fast multipole method (Coulomb kernel).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It is a
 * plain, slow, obviously-correct restatement of the method in double
 * precision and shares no code with the CUDA path.
 *
 * What it covers (paper sections / equations):
 *   - numerical DA (truncated power series algebra) in three variables:
 *     Appendix A (addition, multiplication, derivation, inverse and roots of
 *     elements that are not infinitely small, composition);
 *   - the seven operators P2M (Eq. 1-2), M2M (Eq. 3-4), M2L (Eq. 5),
 *     P2L (Eq. 6), L2L (Eq. 7), L2P and M2P (Sec. 3.2 evaluation);
 *   - the pairwise direct sum (Eq. 1) with compensated summation;
 *   - the octree (uniform, or adaptive with leaf size s, Sec. 3.5) and the
 *     U/V/W/X interaction lists of the adaptive FMM of Cheng, Greengard and
 *     Rokhlin (J. Comput. Phys. 155, 1999), which the paper's framework uses
 *     (Sec. 1; Sec. 3.4: at most 189 M2L partners per box);
 *   - the FMM traversal of Sec. 1.
 *
 * Readings of the paper's garbled or silent passages (all listed in the
 * design notes of the repository):
 *   - Eq. 2: the cross term is -2 r_i.d (the printed "+" gives the
 *     potential of the mirrored charge);
 *   - Eq. 5: R = 1/|r0+r'|^2, so that d = r/r^2 and sqrt(R) = |d|;
 *   - fields are E = -grad(phi), from a first-order DA in the target offset;
 *   - j == i and coincident points (r = 0) are skipped in every pair sum.
 *
 * Conventions: coefficient index of d^(a,b,c) is graded by total order
 * n = a+b+c; inside an order, the x exponent descends, then the y exponent
 * (Table 1 shows this order).  All arrays are caller-owned, row-major.
 * Functions return 0 on success and a negative code on bad arguments.
 */
#ifndef DAFMM_ORACLE_H
#define DAFMM_ORACLE_H
#include <stdint.h>

#define OR_MAXORD 12

#ifdef __cplusplus
extern "C" {
#endif

/* ---- numerical DA (Appendix A) ---------------------------------------- */
int    or_ncoef(int order);
/* exponents of coefficient i: out[0..2] */
int    or_exponents(int order, int i, int* out3);
/* truncated product c = a*b */
int    or_da_mul(int order, const double* a, const double* b, double* c);
/* c = a^s by the binomial series in (a - a0)/a0; requires a0 > 0 */
int    or_da_pow(int order, const double* a, double s, double* c);
/* derivation d/dx_v (v = 0,1,2), result truncated at order-1 (stored in the same layout) */
int    or_da_deriv(int order, const double* a, int v, double* c);
/* f o g: f has order fo, g[3] (each ncoef(go) long, packed) have order go; result has order go */
int    or_da_compose(int fo, const double* f, int go, const double* g, double* out);
double or_da_eval(int order, const double* a, const double* x3);
/* DA vector of 1/|x0 + d| about the point x0 (Table 1 computes it at (1,1,1), order 2) */
int    or_da_rinv(int order, const double* x0, double* out);

/* ---- the seven operators ---------------------------------------------- */
/* P2M, Eq. 2: M += sum_i q_i (1 - 2 s_i.d + s_i^2 d^2)^(-1/2); s = n x 3 offsets from the box centre */
int or_p2m(int order, int64_t n, const double* s, const double* q, double* M);
/* M2M, Eq. 3-4: out += sqrt(R) (M o M1); r0 = parent centre - child centre */
int or_m2m(int order, const double* M, const double* r0, double* out);
/* M2L, Eq. 5 by DA composition: out += sqrt(R) (M o M2); r0 = target centre - source centre */
int or_m2l(int order, const double* M, const double* r0, double* out);
/* M2L by rotation (Sec. 3.4): rotate M so that r0 lies on the positive x axis, apply Eq. 5
 * along the axis, rotate the result back; equal to or_m2l up to rounding */
int or_m2l_rot(int order, const double* M, const double* r0, double* out);
/* the rotation of Sec. 3.4 (about x by atan2(z, y), then about z by atan2(sqrt(y^2+z^2), x)):
 * Q (3x3 row-major) with Q r0 = (|r0|, 0, 0) */
int or_rotation(const double* r0, double* Q9);
/* out = a o (u -> A u), A 3x3 row-major */
int or_da_linmap(int order, const double* a, const double* A9, double* out);
/* the M2L transfer map of Eq. 5: sqrt(R) and the three components of M2 (packed) */
int or_m2l_map(int order, const double* r0, double* sqrtR, double* map3);
/* M2L as a matrix: K[beta*nc + alpha] = coefficient beta of M2L(e_alpha); exact by linearity */
int or_m2l_matrix(int order, const double* r0, double* K);
/* P2L, Eq. 6: L += sum_i q_i / |w_i + d'|, w_i = (target centre - source position)_i (n x 3) */
int or_p2l(int order, int64_t n, const double* w, const double* q, double* L);
/* L2L, Eq. 7: out += L o (r0 + d'); r0 = child centre - parent centre */
int or_l2l(int order, const double* L, const double* r0, double* out);
/* L2P: phi_i += L(x_i), field_i += -grad L(x_i); x = n x 3 offsets from the box centre */
int or_l2p(int order, const double* L, int64_t n, const double* x, double* phi, double* field);
/* M2P: phi_i += |d| M(d), d = s/|s|^2; field_i += -grad_s; s = n x 3 offsets from the source centre */
int or_m2p(int order, const double* M, int64_t n, const double* s, double* phi, double* field);

/* ---- direct sum, Eq. 1 -------------------------------------------------- */
/* phi_t = sum_{j != t, r>0} q_j/r, field_t = sum q_j (r_t - r_j)/r^3 for targets t in tgt[0..nt)
 * (tgt == NULL: all n targets, in order).  Neumaier-compensated sums. */
int or_direct(int64_t n, const double* xyz, const double* q, int64_t nt, const int64_t* tgt,
              double* phi, double* field, int nthreads);

/* ---- octree and interaction lists --------------------------------------- */
typedef struct or_tree or_tree;
/* domain = {x0, y0, z0, size}; uniform_depth >= 0 builds a uniform tree of that depth,
 * otherwise boxes with more than max_leaf particles split, up to max_depth (<= 21). */
or_tree* or_tree_build(int64_t n, const double* xyz, const double* domain4,
                       int uniform_depth, int max_leaf, int max_depth);
void     or_tree_free(or_tree* t);
int      or_tree_nbox(const or_tree* t);
/* per box: level, ijk[3], parent, is_leaf, particle begin/end in the sorted order */
int      or_tree_box(const or_tree* t, int b, int64_t* info8);
/* sorted order of particles: perm[k] = original index of the k-th sorted particle */
int      or_tree_perm(const or_tree* t, int64_t* perm);
/* list = 0:U 1:V 2:W 3:X; returns count, writes up to cap entries */
int      or_tree_list(const or_tree* t, int b, int list, int* out, int cap);

/* ---- FMM traversal (Sec. 1) --------------------------------------------- */
/* m2l_mode: 0 = DA composition per pair (Eq. 5 literally), 1 = matrices cached per (level, v),
 * 2 = the rotation-based M2L of Sec. 3.4 per pair (M2M and L2L as in mode 0).
 * tgt: NULL for all targets, else only those targets are computed (outputs in tgt order). */
int or_fmm(int64_t n, const double* xyz, const double* q, const double* domain4,
           int uniform_depth, int max_leaf, int max_depth, int order, int m2l_mode,
           int64_t nt, const int64_t* tgt, double* phi, double* field, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
