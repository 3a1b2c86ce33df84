/*
 * ops.c -- the seven DA-FMM operators for the Coulomb kernel, written as the
 * paper's equations in numerical DA arithmetic (Sec. 2).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle_internal.h"

/* the DA vector of the basis variable d_v (plus a constant c0) */
static void da_var(const tpsa_ctx* t, double* a, int v, double c0) {
    da_const(t, a, c0);
    if (t->order >= 1) a[tpsa_index(v == 0, v == 1, v == 2)] = 1.0;
}

/* d.d as a DA vector */
static void da_dd(const tpsa_ctx* t, double* a) {
    da_zero(t, a);
    if (t->order >= 2) {
        a[tpsa_index(2, 0, 0)] = 1.0;
        a[tpsa_index(0, 2, 0)] = 1.0;
        a[tpsa_index(0, 0, 2)] = 1.0;
    }
}

/* P2M, Eq. 2 (Sec. 2.1): with d = r/r^2,
 *   phi = sum_i q_i/|r_i - r| = |d| sum_i q_i (1 + r_i^2 d^2 - 2 r_i.d)^(-1/2).
 * The cross term carries a minus sign: |r - r_i|^2 = r^2 (1 - 2 r_i.d + r_i^2 d^2). */
void op_p2m1(const tpsa_ctx* t, const double* s, double q, double* M) {
    double v[TPSA_MAXCOEF], dd[TPSA_MAXCOEF], r[TPSA_MAXCOEF];
    double s2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    da_dd(t, dd);
    da_const(t, v, 1.0);
    if (t->order >= 1)
        for (int k = 0; k < 3; ++k) v[tpsa_index(k == 0, k == 1, k == 2)] = -2.0 * s[k];
    da_axpy(t, s2, dd, v);
    da_pow(t, v, -0.5, r);
    da_axpy(t, q, r, M);
}

/* M2M, Eq. 3-4 (Sec. 2.2): child centre at the origin, parent centre r0,
 *   M1: d = (d' + d'^2 r0) R,  R = 1/(1 + r0^2 d'^2 + 2 r0.d'),
 *   M' = sqrt(R) (M o M1). */
void op_m2m(const tpsa_ctx* t, const double* M, const double* r0, double* out) {
    double u[TPSA_MAXCOEF], R[TPSA_MAXCOEF], sR[TPSA_MAXCOEF], dd[TPSA_MAXCOEF];
    double map[3][TPSA_MAXCOEF], tmp[TPSA_MAXCOEF], comp[TPSA_MAXCOEF];
    double r02 = r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2];
    da_dd(t, dd);
    da_const(t, u, 1.0);
    da_axpy(t, r02, dd, u);
    if (t->order >= 1)
        for (int k = 0; k < 3; ++k) u[tpsa_index(k == 0, k == 1, k == 2)] += 2.0 * r0[k];
    da_pow(t, u, -1.0, R);
    da_pow(t, u, -0.5, sR);
    for (int k = 0; k < 3; ++k) {
        da_var(t, tmp, k, 0.0);
        da_axpy(t, r0[k], dd, tmp);
        da_mul(t, tmp, R, map[k]);
    }
    const double* g[3] = {map[0], map[1], map[2]};
    da_compose(t, M, t, g, comp);
    da_mul(t, sR, comp, tmp);
    da_axpy(t, 1.0, tmp, out);
}

/* M2L transfer map, Eq. 5 (Sec. 2.3): source centre at the origin, target centre r0,
 *   M2: d = (r0 + d') R,  R = 1/|r0 + d'|^2  (so that sqrt(R) = |d|). */
void op_m2l_map(const tpsa_ctx* t, const double* r0, double* sqrtR, double* map3) {
    double w[3][TPSA_MAXCOEF], u[TPSA_MAXCOEF], sq[TPSA_MAXCOEF], R[TPSA_MAXCOEF];
    da_zero(t, u);
    for (int k = 0; k < 3; ++k) {
        da_var(t, w[k], k, r0[k]);
        da_mul(t, w[k], w[k], sq);
        da_axpy(t, 1.0, sq, u);
    }
    da_pow(t, u, -1.0, R);
    da_pow(t, u, -0.5, sqrtR);
    for (int k = 0; k < 3; ++k) da_mul(t, w[k], R, map3 + (size_t)k * t->ncoef);
}

/* M2L, Eq. 5: phi_L = sqrt(R) (phi_M o M2) */
void op_m2l(const tpsa_ctx* t, const double* M, const double* r0, double* out) {
    double sR[TPSA_MAXCOEF], map[3 * TPSA_MAXCOEF], comp[TPSA_MAXCOEF], tmp[TPSA_MAXCOEF];
    op_m2l_map(t, r0, sR, map);
    const double* g[3] = {map, map + t->ncoef, map + 2 * t->ncoef};
    da_compose(t, M, t, g, comp);
    da_mul(t, sR, comp, tmp);
    da_axpy(t, 1.0, tmp, out);
}

/* The rotation of Sec. 3.4 that puts r0 on the positive x axis: first about the x axis by
 * theta = atan2(z, y), which brings r0 into the x-y plane, then about the z axis by
 * phi = atan2(sqrt(y^2 + z^2), x).  Q = Rz(phi) Rx(theta) (row-major), Q r0 = (|r0|, 0, 0).
 * With y = z = 0 the first rotation is the identity. */
void op_rotation(const double* r0, double* Q) {
    const double x = r0[0], y = r0[1], z = r0[2];
    const double ryz = sqrt(y * y + z * z), rho = sqrt(x * x + y * y + z * z);
    const double c1 = ryz > 0.0 ? y / ryz : 1.0, s1 = ryz > 0.0 ? z / ryz : 0.0;
    const double c2 = rho > 0.0 ? x / rho : 1.0, s2 = rho > 0.0 ? ryz / rho : 0.0;
    /* Rx = [[1,0,0],[0,c1,s1],[0,-s1,c1]], Rz = [[c2,s2,0],[-s2,c2,0],[0,0,1]] */
    const double Rx[9] = {1, 0, 0, 0, c1, s1, 0, -s1, c1};
    const double Rz[9] = {c2, s2, 0, -s2, c2, 0, 0, 0, 1};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += Rz[3 * i + k] * Rx[3 * k + j];
            Q[3 * i + j] = v;
        }
}

/* a o (u -> A u): the DA vector a composed with the linear map of the 3x3 matrix A
 * (row-major), i.e. the map whose components are u_i -> sum_j A_ij u_j */
void op_linmap(const tpsa_ctx* t, const double* a, const double* A, double* out) {
    double map[3][TPSA_MAXCOEF];
    for (int i = 0; i < 3; ++i) {
        da_zero(t, map[i]);
        if (t->order >= 1)
            for (int j = 0; j < 3; ++j) map[i][tpsa_index(j == 0, j == 1, j == 2)] = A[3 * i + j];
    }
    const double* g[3] = {map[0], map[1], map[2]};
    da_compose(t, a, t, g, out);
}

/* M2L by rotation (Sec. 3.4): with Q r0 = (|r0|, 0, 0) and u = Q d, the source expansion in
 * the rotated variables is M^(u) = M(Q^T u); Eq. 5 along the axis gives
 * L^(e) = sqrt(R(e)) M^(M2(e)) for r0' = (|r0|, 0, 0); the result in the target variables
 * is L(d') = L^(Q d'). */
void op_m2l_rot(const tpsa_ctx* t, const double* M, const double* r0, double* out) {
    double Q[9], Qt[9], Mh[TPSA_MAXCOEF], Lh[TPSA_MAXCOEF], L[TPSA_MAXCOEF];
    op_rotation(r0, Q);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Qt[3 * i + j] = Q[3 * j + i];
    const double ax[3] = {sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]), 0.0, 0.0};
    op_linmap(t, M, Qt, Mh);
    da_zero(t, Lh);
    op_m2l(t, Mh, ax, Lh);
    op_linmap(t, Lh, Q, L);
    da_axpy(t, 1.0, L, out);
}

/* P2L, Eq. 6 (Sec. 2.4): phi_L(d') = q / |r0 - r_i + d'|, w = r0 - r_i */
void op_p2l1(const tpsa_ctx* t, const double* w, double q, double* L) {
    double wv[TPSA_MAXCOEF], sq[TPSA_MAXCOEF], u[TPSA_MAXCOEF], r[TPSA_MAXCOEF];
    da_zero(t, u);
    for (int k = 0; k < 3; ++k) {
        da_var(t, wv, k, w[k]);
        da_mul(t, wv, wv, sq);
        da_axpy(t, 1.0, sq, u);
    }
    da_pow(t, u, -0.5, r);
    da_axpy(t, q, r, L);
}

/* L2L, Eq. 7 (Sec. 2.5): phi_L' = phi_L o M3, M3: d = r0 + d' (parent centre at the origin) */
void op_l2l(const tpsa_ctx* t, const double* L, const double* r0, double* out) {
    double map[3][TPSA_MAXCOEF], comp[TPSA_MAXCOEF];
    for (int k = 0; k < 3; ++k) da_var(t, map[k], k, r0[k]);
    const double* g[3] = {map[0], map[1], map[2]};
    da_compose(t, L, t, g, comp);
    da_axpy(t, 1.0, comp, out);
}

/* L2P (Sec. 3.2): evaluate phi_L at d' = x; the field is read from a first-order DA
 * in the target offset delta: phi_L(x + delta) = phi + grad.delta + O(delta^2). */
void op_l2p1(const tpsa_ctx* t, const double* L, const double* x, double* phi, double* grad) {
    const tpsa_ctx* t1 = tpsa_get(1);
    double map[3][4], res[4];
    for (int k = 0; k < 3; ++k) da_var(t1, map[k], k, x[k]);
    const double* g[3] = {map[0], map[1], map[2]};
    da_compose(t, L, t1, g, res);
    *phi = res[0];
    grad[0] = res[1]; grad[1] = res[2]; grad[2] = res[3];
}

/* M2P (Sec. 3.2): phi = |d| phi_M(d), d = s/|s|^2, s = target - source centre,
 * evaluated in a first-order DA in the target offset. */
void op_m2p1(const tpsa_ctx* t, const double* M, const double* s, double* phi, double* grad) {
    const tpsa_ctx* t1 = tpsa_get(1);
    double sv[3][4], sq[4], u[4], R[4], dv[3][4], dd[4], nd[4], comp[4], res[4];
    da_zero(t1, u);
    for (int k = 0; k < 3; ++k) {
        da_var(t1, sv[k], k, s[k]);
        da_mul(t1, sv[k], sv[k], sq);
        da_axpy(t1, 1.0, sq, u);
    }
    da_pow(t1, u, -1.0, R);
    da_zero(t1, dd);
    for (int k = 0; k < 3; ++k) {
        da_mul(t1, sv[k], R, dv[k]);
        da_mul(t1, dv[k], dv[k], sq);
        da_axpy(t1, 1.0, sq, dd);
    }
    da_pow(t1, dd, 0.5, nd);
    const double* g[3] = {dv[0], dv[1], dv[2]};
    da_compose(t, M, t1, g, comp);
    da_mul(t1, nd, comp, res);
    *phi = res[0];
    grad[0] = res[1]; grad[1] = res[2]; grad[2] = res[3];
}

/* ---- exported batch wrappers ------------------------------------------------ */
int or_p2m(int order, int64_t n, const double* s, const double* q, double* M) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t || n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) op_p2m1(t, s + 3 * i, q[i], M);
    return 0;
}

int or_m2m(int order, const double* M, const double* r0, double* out) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    op_m2m(t, M, r0, out);
    return 0;
}

int or_m2l(int order, const double* M, const double* r0, double* out) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    op_m2l(t, M, r0, out);
    return 0;
}

int or_m2l_rot(int order, const double* M, const double* r0, double* out) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    op_m2l_rot(t, M, r0, out);
    return 0;
}

int or_rotation(const double* r0, double* Q9) {
    if (!r0 || !Q9) return -1;
    op_rotation(r0, Q9);
    return 0;
}

int or_da_linmap(int order, const double* a, const double* A9, double* out) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    op_linmap(t, a, A9, out);
    return 0;
}

int or_m2l_map(int order, const double* r0, double* sqrtR, double* map3) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    op_m2l_map(t, r0, sqrtR, map3);
    return 0;
}

int or_m2l_matrix(int order, const double* r0, double* K) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    int nc = t->ncoef;
    double sR[TPSA_MAXCOEF], map[3 * TPSA_MAXCOEF], col[TPSA_MAXCOEF];
    op_m2l_map(t, r0, sR, map);
    const double* g[3] = {map, map + nc, map + 2 * nc};
    double* mono = (double*)malloc(sizeof(double) * (size_t)nc * nc);
    da_monomials(t, t, g, mono);
    for (int a = 0; a < nc; ++a) {
        da_mul(t, sR, mono + (size_t)a * nc, col);
        for (int b = 0; b < nc; ++b) K[(size_t)b * nc + a] = col[b];
    }
    free(mono);
    return 0;
}

int or_p2l(int order, int64_t n, const double* w, const double* q, double* L) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t || n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) op_p2l1(t, w + 3 * i, q[i], L);
    return 0;
}

int or_l2l(int order, const double* L, const double* r0, double* out) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    op_l2l(t, L, r0, out);
    return 0;
}

int or_l2p(int order, const double* L, int64_t n, const double* x, double* phi, double* field) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t || n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        double p, g[3];
        op_l2p1(t, L, x + 3 * i, &p, g);
        phi[i] += p;
        for (int k = 0; k < 3; ++k) field[3 * i + k] -= g[k];
    }
    return 0;
}

int or_m2p(int order, const double* M, int64_t n, const double* s, double* phi, double* field) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t || n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        double p, g[3];
        op_m2p1(t, M, s + 3 * i, &p, g);
        phi[i] += p;
        for (int k = 0; k < 3; ++k) field[3 * i + k] -= g[k];
    }
    return 0;
}
