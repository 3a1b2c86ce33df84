/*
 * tpsa.c -- numerical DA vectors in three variables (paper, Appendix A and Sec. 2).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * A DA vector of order p stores the coefficient of every monomial
 * d1^a d2^b d3^c with a+b+c <= p (Eq. A.5: [a] = sum c_J d^J).  The
 * arithmetic below is the textbook one:
 *   - product: full polynomial product, truncated above order p (Eq. A.1);
 *   - derivation: d/dx_v of the polynomial, which drops to order p-1 (Eq. A.2);
 *   - a^s for an element that is not infinitely small (a0 > 0): write
 *     a = a0 (1 + t), t = (a - a0)/a0 nilpotent, then
 *     a^s = a0^s sum_{k=0..p} binom(s,k) t^k (fixed-point theorem, App. A;
 *     s = -1 is the inverse, s = 1/2 the root);
 *   - composition f o g: evaluate the polynomial f with DA arithmetic at the
 *     DA vectors g (Sec. 2 "composition of two functions").
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle_internal.h"

static tpsa_ctx g_ctx[OR_MAXORD + 1];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

int tpsa_index(int a, int b, int c) {
    int n = a + b + c;
    /* number of monomials of order < n, then position inside order n:
       exponents of x descend, then exponents of y descend */
    return n * (n + 1) * (n + 2) / 6 + (n - a) * (n - a + 1) / 2 + c;
}

static void init_ctx(tpsa_ctx* t, int p) {
    t->order = p;
    t->ncoef = (p + 1) * (p + 2) * (p + 3) / 6;
    t->e = (int(*)[3])malloc(sizeof(int[3]) * t->ncoef);
    t->ord = (int*)malloc(sizeof(int) * t->ncoef);
    for (int n = 0; n <= p; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                int c = n - a - b;
                int i = tpsa_index(a, b, c);
                t->e[i][0] = a; t->e[i][1] = b; t->e[i][2] = c;
                t->ord[i] = n;
            }
    /* product table: every pair (i, j) with ord(i)+ord(j) <= p and its target k */
    int cnt = 0;
    for (int i = 0; i < t->ncoef; ++i)
        for (int j = 0; j < t->ncoef; ++j)
            if (t->ord[i] + t->ord[j] <= p) ++cnt;
    t->nmul = cnt;
    t->mul = (int(*)[3])malloc(sizeof(int[3]) * (cnt > 0 ? cnt : 1));
    /* rows grouped by i so that a zero left factor can skip its whole row */
    t->row = (int*)malloc(sizeof(int) * (t->ncoef + 1));
    cnt = 0;
    for (int i = 0; i < t->ncoef; ++i) {
        t->row[i] = cnt;
        for (int j = 0; j < t->ncoef; ++j)
            if (t->ord[i] + t->ord[j] <= p) {
                t->mul[cnt][0] = i;
                t->mul[cnt][1] = j;
                t->mul[cnt][2] = tpsa_index(t->e[i][0] + t->e[j][0], t->e[i][1] + t->e[j][1],
                                            t->e[i][2] + t->e[j][2]);
                ++cnt;
            }
    }
    t->row[t->ncoef] = cnt;
}

static void init_all(void) {
    for (int p = 0; p <= OR_MAXORD; ++p) init_ctx(&g_ctx[p], p);
}

const tpsa_ctx* tpsa_get(int order) {
    if (order < 0 || order > OR_MAXORD) return NULL;
    pthread_once(&g_once, init_all);
    return &g_ctx[order];
}

void da_zero(const tpsa_ctx* t, double* a) { memset(a, 0, sizeof(double) * t->ncoef); }

void da_const(const tpsa_ctx* t, double* a, double c) { da_zero(t, a); a[0] = c; }

void da_copy(const tpsa_ctx* t, const double* a, double* c) { memcpy(c, a, sizeof(double) * t->ncoef); }

void da_axpy(const tpsa_ctx* t, double s, const double* a, double* c) {
    for (int i = 0; i < t->ncoef; ++i) c[i] += s * a[i];
}

void da_mul(const tpsa_ctx* t, const double* a, const double* b, double* c) {
    double tmp[TPSA_MAXCOEF];
    memset(tmp, 0, sizeof(double) * t->ncoef);
    for (int i = 0; i < t->ncoef; ++i) {
        if (a[i] == 0.0) continue;
        for (int m = t->row[i]; m < t->row[i + 1]; ++m) tmp[t->mul[m][2]] += a[i] * b[t->mul[m][1]];
    }
    memcpy(c, tmp, sizeof(double) * t->ncoef);
}

int da_pow(const tpsa_ctx* t, const double* a, double s, double* c) {
    double a0 = a[0];
    if (!(a0 > 0.0)) return -1;
    double tv[TPSA_MAXCOEF], term[TPSA_MAXCOEF], acc[TPSA_MAXCOEF];
    /* t = (a - a0)/a0, no constant part */
    for (int i = 0; i < t->ncoef; ++i) tv[i] = a[i] / a0;
    tv[0] = 0.0;
    da_const(t, term, 1.0);
    da_const(t, acc, 1.0);
    double binom = 1.0;
    for (int k = 1; k <= t->order; ++k) {
        binom = binom * (s - (double)(k - 1)) / (double)k;
        da_mul(t, tv, term, term);
        da_axpy(t, binom, term, acc);
    }
    double scale = pow(a0, s);
    for (int i = 0; i < t->ncoef; ++i) c[i] = scale * acc[i];
    return 0;
}

void da_deriv(const tpsa_ctx* t, const double* a, int v, double* c) {
    double tmp[TPSA_MAXCOEF];
    memset(tmp, 0, sizeof(double) * t->ncoef);
    for (int i = 0; i < t->ncoef; ++i) {
        int e[3] = {t->e[i][0], t->e[i][1], t->e[i][2]};
        if (e[v] == 0) continue;
        double f = (double)e[v];
        e[v] -= 1;
        tmp[tpsa_index(e[0], e[1], e[2])] += f * a[i];
    }
    memcpy(c, tmp, sizeof(double) * t->ncoef);
}

double da_eval(const tpsa_ctx* t, const double* a, const double* x) {
    double s = 0.0;
    for (int i = 0; i < t->ncoef; ++i) {
        double m = a[i];
        for (int k = 0; k < t->e[i][0]; ++k) m *= x[0];
        for (int k = 0; k < t->e[i][1]; ++k) m *= x[1];
        for (int k = 0; k < t->e[i][2]; ++k) m *= x[2];
        s += m;
    }
    return s;
}

/* monomials g^alpha for every alpha of order <= tf->order, in tg arithmetic.
   mono must hold tf->ncoef * tg->ncoef doubles. */
void da_monomials(const tpsa_ctx* tf, const tpsa_ctx* tg, const double* const g[3], double* mono) {
    int ng = tg->ncoef;
    da_const(tg, mono, 1.0);
    for (int i = 1; i < tf->ncoef; ++i) {
        int e[3] = {tf->e[i][0], tf->e[i][1], tf->e[i][2]};
        int v = (e[0] > 0) ? 0 : (e[1] > 0 ? 1 : 2);
        e[v] -= 1;
        int prev = tpsa_index(e[0], e[1], e[2]);
        da_mul(tg, g[v], mono + (size_t)prev * ng, mono + (size_t)i * ng);
    }
}

void da_compose(const tpsa_ctx* tf, const double* f, const tpsa_ctx* tg, const double* const g[3],
                double* out) {
    int ng = tg->ncoef;
    double* mono = (double*)malloc(sizeof(double) * (size_t)tf->ncoef * ng);
    da_monomials(tf, tg, g, mono);
    da_zero(tg, out);
    for (int i = 0; i < tf->ncoef; ++i)
        if (f[i] != 0.0) da_axpy(tg, f[i], mono + (size_t)i * ng, out);
    free(mono);
}

/* ---- exported wrappers ---------------------------------------------------- */
int or_ncoef(int order) {
    const tpsa_ctx* t = tpsa_get(order);
    return t ? t->ncoef : -1;
}

int or_exponents(int order, int i, int* out3) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t || i < 0 || i >= t->ncoef) return -1;
    out3[0] = t->e[i][0]; out3[1] = t->e[i][1]; out3[2] = t->e[i][2];
    return 0;
}

int or_da_mul(int order, const double* a, const double* b, double* c) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    da_mul(t, a, b, c);
    return 0;
}

int or_da_pow(int order, const double* a, double s, double* c) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    return da_pow(t, a, s, c);
}

int or_da_deriv(int order, const double* a, int v, double* c) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t || v < 0 || v > 2) return -1;
    da_deriv(t, a, v, c);
    return 0;
}

int or_da_compose(int fo, const double* f, int go, const double* g, double* out) {
    const tpsa_ctx* tf = tpsa_get(fo);
    const tpsa_ctx* tg = tpsa_get(go);
    if (!tf || !tg) return -1;
    const double* gv[3] = {g, g + tg->ncoef, g + 2 * tg->ncoef};
    da_compose(tf, f, tg, gv, out);
    return 0;
}

double or_da_eval(int order, const double* a, const double* x3) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return NAN;
    return da_eval(t, a, x3);
}

int or_da_rinv(int order, const double* x0, double* out) {
    const tpsa_ctx* t = tpsa_get(order);
    if (!t) return -1;
    /* v = (x+d1)^2 + (y+d2)^2 + (z+d3)^2 built from DA products, then v^(-1/2) */
    double w[TPSA_MAXCOEF], sq[TPSA_MAXCOEF], v[TPSA_MAXCOEF];
    da_zero(t, v);
    for (int k = 0; k < 3; ++k) {
        da_const(t, w, x0[k]);
        if (t->order >= 1) w[tpsa_index(k == 0, k == 1, k == 2)] = 1.0;
        da_mul(t, w, w, sq);
        da_axpy(t, 1.0, sq, v);
    }
    return da_pow(t, v, -0.5, out);
}
