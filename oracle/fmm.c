/*
 * fmm.c -- the FMM traversal of Sec. 1 on the oracle's octree:
 *   P2M at leaves -> M2M upward -> M2L over V lists (+ P2L over X lists)
 *   -> L2L downward -> L2P (+ M2P over W lists) + P2P over U lists.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Displacements between box centres are formed from the integer box
 * coordinates (exact multiples of the box width), particle offsets as
 * x - centre in double precision.
 *
 * m2l_mode 0 applies Eq. 5 by DA composition for every pair; m2l_mode 1
 * applies the same linear maps as matrices whose columns are the operator
 * applied to unit vectors (exact by linearity), cached per level and
 * displacement for M2L and per level and octant for M2M/L2L; m2l_mode 2 applies
 * the rotation-based M2L of Sec. 3.4 for every pair (M2M and L2L as in mode 0).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle_internal.h"
#include "tree_internal.h"

typedef struct {
    const or_tree* t;
    const tpsa_ctx* ctx;
    int nc, mode;
    const double *xyz, *q;
    double *M, *L;         /* nbox x nc */
    char* need;            /* boxes whose local expansion is needed */
    int64_t* outpos;       /* particle -> output slot, or -1 */
    double *phi, *field;
    int level;
    double** Kcache;       /* 343 per level (M2L), index (dx+3)*49+(dy+3)*7+(dz+3) */
    double** Scache;       /* 8 M2M and 8 L2L matrices for the current level */
} fmm_ctx;

static double box_width(const or_tree* t, int level) { return ldexp(t->dom[3], -level); }

static void box_centre(const or_tree* t, int b, double* c) {
    double h = box_width(t, t->box[b].level);
    for (int d = 0; d < 3; ++d) c[d] = t->dom[d] + ((double)t->box[b].ijk[d] + 0.5) * h;
}

static void matvec_acc(int nc, const double* K, const double* x, double* y) {
    for (int b = 0; b < nc; ++b) {
        double s = 0.0;
        const double* row = K + (size_t)b * nc;
        for (int a = 0; a < nc; ++a) s += row[a] * x[a];
        y[b] += s;
    }
}

/* ---- P2M at leaves ---- */
static void p2m_range(int64_t b0, int64_t b1, void* p) {
    fmm_ctx* f = (fmm_ctx*)p;
    const or_tree* t = f->t;
    for (int64_t b = b0; b < b1; ++b) {
        if (!t->box[b].is_leaf) continue;
        double c[3];
        box_centre(t, (int)b, c);
        for (int64_t k = t->box[b].pbeg; k < t->box[b].pend; ++k) {
            int64_t i = t->perm[k];
            double s[3] = {f->xyz[3 * i] - c[0], f->xyz[3 * i + 1] - c[1], f->xyz[3 * i + 2] - c[2]};
            op_p2m1(f->ctx, s, f->q[i], f->M + (size_t)b * f->nc);
        }
    }
}

/* ---- M2M for the parents at level f->level ---- */
static void m2m_range(int64_t b0, int64_t b1, void* p) {
    fmm_ctx* f = (fmm_ctx*)p;
    const or_tree* t = f->t;
    for (int64_t b = b0; b < b1; ++b) {
        if (t->box[b].level != f->level || t->box[b].is_leaf) continue;
        double hc = box_width(t, f->level + 1);
        for (int c = 0; c < 8; ++c) {
            int ch = t->box[b].child[c];
            if (ch < 0) continue;
            double r0[3];
            for (int d = 0; d < 3; ++d)
                r0[d] = ((double)(2 * t->box[b].ijk[d] - t->box[ch].ijk[d]) + 0.5) * hc;
            if (f->mode != 1) op_m2m(f->ctx, f->M + (size_t)ch * f->nc, r0, f->M + (size_t)b * f->nc);
            else matvec_acc(f->nc, f->Scache[c], f->M + (size_t)ch * f->nc, f->M + (size_t)b * f->nc);
        }
    }
}

/* ---- M2L (V list) and P2L (X list) into boxes of level f->level ---- */
static void m2l_range(int64_t b0, int64_t b1, void* p) {
    fmm_ctx* f = (fmm_ctx*)p;
    const or_tree* t = f->t;
    for (int64_t b = b0; b < b1; ++b) {
        if (t->box[b].level != f->level || !f->need[b]) continue;
        double h = box_width(t, f->level);
        double* Lb = f->L + (size_t)b * f->nc;
        for (int k = 0; k < t->V[b].n; ++k) {
            int c = t->V[b].a[k];
            int64_t dv[3];
            for (int d = 0; d < 3; ++d) dv[d] = t->box[b].ijk[d] - t->box[c].ijk[d];
            if (f->mode != 1) {
                double r0[3] = {(double)dv[0] * h, (double)dv[1] * h, (double)dv[2] * h};
                if (f->mode == 2) op_m2l_rot(f->ctx, f->M + (size_t)c * f->nc, r0, Lb);
                else op_m2l(f->ctx, f->M + (size_t)c * f->nc, r0, Lb);
            } else {
                int key = (int)((dv[0] + 3) * 49 + (dv[1] + 3) * 7 + (dv[2] + 3));
                matvec_acc(f->nc, f->Kcache[key], f->M + (size_t)c * f->nc, Lb);
            }
        }
        double cb[3];
        box_centre(t, (int)b, cb);
        for (int k = 0; k < t->X[b].n; ++k) {
            int c = t->X[b].a[k];
            for (int64_t j = t->box[c].pbeg; j < t->box[c].pend; ++j) {
                int64_t i = t->perm[j];
                double w[3] = {cb[0] - f->xyz[3 * i], cb[1] - f->xyz[3 * i + 1], cb[2] - f->xyz[3 * i + 2]};
                op_p2l1(f->ctx, w, f->q[i], Lb);
            }
        }
    }
}

/* ---- L2L into boxes of level f->level ---- */
static void l2l_range(int64_t b0, int64_t b1, void* p) {
    fmm_ctx* f = (fmm_ctx*)p;
    const or_tree* t = f->t;
    for (int64_t b = b0; b < b1; ++b) {
        if (t->box[b].level != f->level || !f->need[b]) continue;
        int P = t->box[b].parent;
        double hc = box_width(t, f->level);
        int c = (int)((t->box[b].ijk[0] & 1) | ((t->box[b].ijk[1] & 1) << 1) | ((t->box[b].ijk[2] & 1) << 2));
        if (f->mode != 1) {
            double r0[3];
            for (int d = 0; d < 3; ++d)
                r0[d] = ((double)(t->box[b].ijk[d] - 2 * t->box[P].ijk[d]) - 0.5) * hc;
            op_l2l(f->ctx, f->L + (size_t)P * f->nc, r0, f->L + (size_t)b * f->nc);
        } else {
            matvec_acc(f->nc, f->Scache[8 + c], f->L + (size_t)P * f->nc, f->L + (size_t)b * f->nc);
        }
    }
}

/* ---- leaves: L2P + M2P (W list) + P2P (U list) ---- */
static void leaf_range(int64_t b0, int64_t b1, void* p) {
    fmm_ctx* f = (fmm_ctx*)p;
    const or_tree* t = f->t;
    for (int64_t b = b0; b < b1; ++b) {
        if (!t->box[b].is_leaf || !f->need[b]) continue;
        double cb[3];
        box_centre(t, (int)b, cb);
        for (int64_t k = t->box[b].pbeg; k < t->box[b].pend; ++k) {
            int64_t i = t->perm[k];
            int64_t o = f->outpos[i];
            if (o < 0) continue;
            const double* ri = f->xyz + 3 * i;
            double ph = 0.0, E[3] = {0, 0, 0}, g[3], pv;
            double x[3] = {ri[0] - cb[0], ri[1] - cb[1], ri[2] - cb[2]};
            op_l2p1(f->ctx, f->L + (size_t)b * f->nc, x, &pv, g);
            ph += pv;
            for (int d = 0; d < 3; ++d) E[d] -= g[d];
            for (int w = 0; w < t->W[b].n; ++w) {
                int c = t->W[b].a[w];
                double cc[3];
                box_centre(t, c, cc);
                double s[3] = {ri[0] - cc[0], ri[1] - cc[1], ri[2] - cc[2]};
                op_m2p1(f->ctx, f->M + (size_t)c * f->nc, s, &pv, g);
                ph += pv;
                for (int d = 0; d < 3; ++d) E[d] -= g[d];
            }
            for (int u = 0; u < t->U[b].n; ++u) {
                int c = t->U[b].a[u];
                for (int64_t m = t->box[c].pbeg; m < t->box[c].pend; ++m) {
                    int64_t j = t->perm[m];
                    if (j == i) continue;
                    double dx = ri[0] - f->xyz[3 * j], dy = ri[1] - f->xyz[3 * j + 1], dz = ri[2] - f->xyz[3 * j + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2);
                    double qr = f->q[j] / r;
                    ph += qr;
                    double qr3 = qr / r2;
                    E[0] += qr3 * dx; E[1] += qr3 * dy; E[2] += qr3 * dz;
                }
            }
            f->phi[o] = ph;
            for (int d = 0; d < 3; ++d) f->field[3 * o + d] = E[d];
        }
    }
}

/* matrices of the M2L maps used at one level */
typedef struct { fmm_ctx* f; int* keys; } kgen_arg;
static void kgen_range(int64_t k0, int64_t k1, void* p) {
    kgen_arg* a = (kgen_arg*)p;
    double h = box_width(a->f->t, a->f->level);
    for (int64_t k = k0; k < k1; ++k) {
        int key = a->keys[k];
        double r0[3] = {(double)(key / 49 - 3) * h, (double)((key / 7) % 7 - 3) * h, (double)(key % 7 - 3) * h};
        a->f->Kcache[key] = (double*)malloc(sizeof(double) * (size_t)a->f->nc * a->f->nc);
        or_m2l_matrix(a->f->ctx->order, r0, a->f->Kcache[key]);
    }
}

/* the 8 M2M (parent at level, children at level+1) and 8 L2L (children at level) matrices */
static void shift_matrices(fmm_ctx* f, int level, int which) {
    int nc = f->nc;
    double e[TPSA_MAXCOEF], col[TPSA_MAXCOEF];
    for (int c = 0; c < 8; ++c) {
        int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double* S = f->Scache[which * 8 + c];
        for (int a = 0; a < nc; ++a) {
            memset(e, 0, sizeof(double) * nc);
            e[a] = 1.0;
            memset(col, 0, sizeof(double) * nc);
            double r0[3];
            if (which == 0) {
                double hc = box_width(f->t, level + 1);
                for (int d = 0; d < 3; ++d) r0[d] = (0.5 - (double)o[d]) * hc;
                op_m2m(f->ctx, e, r0, col);
            } else {
                double hc = box_width(f->t, level);
                for (int d = 0; d < 3; ++d) r0[d] = ((double)o[d] - 0.5) * hc;
                op_l2l(f->ctx, e, r0, col);
            }
            for (int b = 0; b < nc; ++b) S[(size_t)b * nc + a] = col[b];
        }
    }
}

int or_fmm(int64_t n, const double* xyz, const double* q, const double* domain4, int uniform_depth,
           int max_leaf, int max_depth, int order, int m2l_mode, int64_t nt, const int64_t* tgt,
           double* phi, double* field, int nthreads) {
    const tpsa_ctx* ctx = tpsa_get(order);
    if (!ctx || n < 0 || m2l_mode < 0 || m2l_mode > 2) return -1;
    or_tree* t = or_tree_build(n, xyz, domain4, uniform_depth, max_leaf, max_depth);
    if (!t) return -2;
    fmm_ctx f;
    memset(&f, 0, sizeof(f));
    f.t = t; f.ctx = ctx; f.nc = ctx->ncoef; f.mode = m2l_mode; f.xyz = xyz; f.q = q;
    f.phi = phi; f.field = field;
    f.M = (double*)calloc((size_t)t->nbox * f.nc, sizeof(double));
    f.L = (double*)calloc((size_t)t->nbox * f.nc, sizeof(double));
    f.need = (char*)calloc(t->nbox, 1);
    f.outpos = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!tgt) nt = n;
    for (int64_t i = 0; i < n; ++i) f.outpos[i] = tgt ? -1 : i;
    for (int64_t k = 0; tgt && k < nt; ++k) {
        if (tgt[k] < 0 || tgt[k] >= n) { or_tree_free(t); return -1; }
        f.outpos[tgt[k]] = k;
    }
    /* boxes on the ancestor chains of leaves that hold targets */
    for (int b = 0; b < t->nbox; ++b) {
        if (!t->box[b].is_leaf) continue;
        int any = 0;
        for (int64_t k = t->box[b].pbeg; k < t->box[b].pend && !any; ++k) any = f.outpos[t->perm[k]] >= 0;
        for (int a = b; any && a >= 0 && !f.need[a]; a = t->box[a].parent) f.need[a] = 1;
    }
    double* Sbuf = NULL;
    double* Sptr[16];
    if (m2l_mode == 1) {
        Sbuf = (double*)malloc(sizeof(double) * 16 * (size_t)f.nc * f.nc);
        for (int k = 0; k < 16; ++k) Sptr[k] = Sbuf + (size_t)k * f.nc * f.nc;
        f.Scache = Sptr;
    }
    /* upward pass */
    parallel_for(t->nbox, nthreads, p2m_range, &f);
    for (int l = t->maxlev - 1; l >= 0; --l) {
        f.level = l;
        if (m2l_mode == 1) shift_matrices(&f, l, 0);
        parallel_for(t->nbox, nthreads, m2m_range, &f);
    }
    /* transfer + downward pass, level by level: every box of level l-1 holds its
       complete local expansion (M2L, P2L and L2L) before level l shifts it down */
    double* Kc[343];
    for (int l = 0; l <= t->maxlev; ++l) {
        f.level = l;
        if (m2l_mode == 1) {
            char used[343];
            memset(used, 0, sizeof(used));
            memset(Kc, 0, sizeof(Kc));
            for (int b = 0; b < t->nbox; ++b) {
                if (t->box[b].level != l || !f.need[b]) continue;
                for (int k = 0; k < t->V[b].n; ++k) {
                    int c = t->V[b].a[k];
                    int key = (int)((t->box[b].ijk[0] - t->box[c].ijk[0] + 3) * 49 +
                                    (t->box[b].ijk[1] - t->box[c].ijk[1] + 3) * 7 +
                                    (t->box[b].ijk[2] - t->box[c].ijk[2] + 3));
                    used[key] = 1;
                }
            }
            int keys[343], nk = 0;
            for (int k = 0; k < 343; ++k) if (used[k]) keys[nk++] = k;
            f.Kcache = Kc;
            kgen_arg ka = {&f, keys};
            parallel_for(nk, nthreads, kgen_range, &ka);
        }
        parallel_for(t->nbox, nthreads, m2l_range, &f);
        if (m2l_mode == 1) for (int k = 0; k < 343; ++k) free(Kc[k]);
        if (l >= 1) {
            if (m2l_mode == 1) shift_matrices(&f, l, 1);
            parallel_for(t->nbox, nthreads, l2l_range, &f);
        }
    }
    parallel_for(t->nbox, nthreads, leaf_range, &f);
    free(Sbuf);
    free(f.M); free(f.L); free(f.need); free(f.outpos);
    or_tree_free(t);
    return 0;
}
