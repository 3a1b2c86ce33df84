/*
 * tree.c -- octree and interaction lists for the oracle.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Boxes are cubes split recursively (Sec. 1).  A uniform tree splits every
 * box down to a fixed depth; an adaptive tree splits a box while it holds
 * more than s particles (Sec. 3.5, leaf size s).  Empty boxes are never
 * created: they carry no multipole and need no local expansion.
 *
 * Box membership comes from 21-bit integer coordinates
 *   k = clamp(floor((x - x0) * (2^21 / size)), 0, 2^21 - 1)
 * and a box at level l holds the particles whose k >> (21 - l) equals its
 * integer coordinates.
 *
 * Lists (Cheng, Greengard, Rokhlin 1999; adjacency = closed cubes touch):
 *   colleagues(b): same-level boxes adjacent to b;
 *   U(b), b leaf : leaves adjacent to b, and b itself       -> P2P;
 *   V(b)         : children of colleagues(parent(b)) not adjacent to b -> M2L
 *                  (at most 189 per box, Sec. 3.4);
 *   W(b), b leaf : descendants of colleagues(b) not adjacent to b whose
 *                  parent is adjacent to b                  -> M2P;
 *   X(b)         : boxes c with b in W(c)                   -> P2L.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle_internal.h"
#include "tree_internal.h"

#define QBITS 21

static void iv_push(ivec* v, int x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 8;
        v->a = (int*)realloc(v->a, sizeof(int) * v->cap);
    }
    v->a[v->n++] = x;
}

static uint64_t spread3(uint64_t x) {
    uint64_t r = 0;
    for (int b = 0; b < QBITS; ++b) r |= ((x >> b) & 1ull) << (3 * b);
    return r;
}

typedef struct { uint64_t key; int64_t idx; } kidx;
static int kidx_cmp(const void* a, const void* b) {
    const kidx *x = (const kidx*)a, *y = (const kidx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

int tree_touch(const or_tree* t, int a, int b) {
    const obox *A = &t->box[a], *B = &t->box[b];
    int L = A->level > B->level ? A->level : B->level;
    for (int d = 0; d < 3; ++d) {
        int64_t alo = A->ijk[d] << (L - A->level), ahi = (A->ijk[d] + 1) << (L - A->level);
        int64_t blo = B->ijk[d] << (L - B->level), bhi = (B->ijk[d] + 1) << (L - B->level);
        if (alo > bhi || blo > ahi) return 0;
    }
    return 1;
}

static int same_level_adjacent(const obox* A, const obox* B) {
    for (int d = 0; d < 3; ++d) {
        int64_t df = A->ijk[d] - B->ijk[d];
        if (df < -1 || df > 1) return 0;
    }
    return 1;
}

static int new_box(or_tree* t, int level, const int64_t* ijk, int parent, int64_t b, int64_t e) {
    if (t->nbox == t->capbox) {
        t->capbox = t->capbox ? 2 * t->capbox : 64;
        t->box = (obox*)realloc(t->box, sizeof(obox) * t->capbox);
    }
    obox* x = &t->box[t->nbox];
    memset(x, 0, sizeof(obox));
    x->level = level;
    for (int d = 0; d < 3; ++d) x->ijk[d] = ijk[d];
    x->parent = parent;
    for (int c = 0; c < 8; ++c) x->child[c] = -1;
    x->is_leaf = 1;
    x->pbeg = b;
    x->pend = e;
    return t->nbox++;
}

static void collect_u(or_tree* t, int node, int b) {
    if (!tree_touch(t, node, b)) return;
    if (t->box[node].is_leaf) {
        iv_push(&t->U[b], node);
        return;
    }
    for (int c = 0; c < 8; ++c)
        if (t->box[node].child[c] >= 0) collect_u(t, t->box[node].child[c], b);
}

static void collect_w(or_tree* t, int node, int b) {
    /* node is adjacent to b and has children */
    for (int c = 0; c < 8; ++c) {
        int ch = t->box[node].child[c];
        if (ch < 0) continue;
        if (tree_touch(t, ch, b)) {
            if (!t->box[ch].is_leaf) collect_w(t, ch, b);
        } else {
            iv_push(&t->W[b], ch);
        }
    }
}

or_tree* or_tree_build(int64_t n, const double* xyz, const double* domain4, int uniform_depth,
                       int max_leaf, int max_depth) {
    if (n < 0 || !domain4 || !(domain4[3] > 0.0)) return NULL;
    if (uniform_depth > QBITS) return NULL;
    if (uniform_depth < 0 && (max_leaf < 1 || max_depth < 0 || max_depth > QBITS)) return NULL;
    or_tree* t = (or_tree*)calloc(1, sizeof(or_tree));
    t->n = n;
    for (int d = 0; d < 4; ++d) t->dom[d] = domain4[d];
    double scale = ldexp(1.0, QBITS) / domain4[3];
    kidx* ki = (kidx*)malloc(sizeof(kidx) * (n > 0 ? n : 1));
    t->qc = (int64_t*)malloc(sizeof(int64_t) * 3 * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        uint64_t key = 0;
        for (int d = 0; d < 3; ++d) {
            double f = floor((xyz[3 * i + d] - domain4[d]) * scale);
            int64_t k = f < 0.0 ? 0 : (f > (double)((1 << QBITS) - 1) ? (1 << QBITS) - 1 : (int64_t)f);
            t->qc[3 * i + d] = k;
            key |= spread3((uint64_t)k) << d;
        }
        ki[i].key = key;
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(kidx), kidx_cmp);
    t->perm = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) t->perm[i] = ki[i].idx;

    int64_t zero[3] = {0, 0, 0};
    new_box(t, 0, zero, -1, 0, n);
    /* breadth-first: boxes of each level are contiguous */
    for (int cur = 0; cur < t->nbox; ++cur) {
        obox b = t->box[cur];
        int split = uniform_depth >= 0 ? (b.level < uniform_depth)
                                       : (b.pend - b.pbeg > max_leaf && b.level < max_depth);
        if (!split) continue;
        int shift = 3 * (QBITS - b.level - 1);
        int64_t s = b.pbeg;
        for (int c = 0; c < 8; ++c) {
            int64_t e = s;
            while (e < b.pend && (int)((ki[e].key >> shift) & 7u) == c) ++e;
            if (e > s) {
                int64_t ijk[3] = {2 * b.ijk[0] + (c & 1), 2 * b.ijk[1] + ((c >> 1) & 1),
                                  2 * b.ijk[2] + ((c >> 2) & 1)};
                int id = new_box(t, b.level + 1, ijk, cur, s, e);
                t->box[cur].child[c] = id;
                t->box[cur].is_leaf = 0;
            }
            s = e;
        }
    }
    free(ki);
    for (int i = 0; i < t->nbox; ++i)
        if (t->box[i].level > t->maxlev) t->maxlev = t->box[i].level;

    /* colleagues, top-down */
    t->C = (ivec*)calloc(t->nbox, sizeof(ivec));
    t->U = (ivec*)calloc(t->nbox, sizeof(ivec));
    t->V = (ivec*)calloc(t->nbox, sizeof(ivec));
    t->W = (ivec*)calloc(t->nbox, sizeof(ivec));
    t->X = (ivec*)calloc(t->nbox, sizeof(ivec));
    for (int b = 1; b < t->nbox; ++b) {
        int P = t->box[b].parent;
        /* candidates: children of P and of P's colleagues */
        for (int k = -1; k < t->C[P].n; ++k) {
            int Q = k < 0 ? P : t->C[P].a[k];
            for (int c = 0; c < 8; ++c) {
                int ch = t->box[Q].child[c];
                if (ch < 0 || ch == b) continue;
                if (same_level_adjacent(&t->box[ch], &t->box[b])) iv_push(&t->C[b], ch);
                else if (k >= 0) iv_push(&t->V[b], ch);
            }
        }
    }
    for (int b = 0; b < t->nbox; ++b) {
        if (!t->box[b].is_leaf) continue;
        collect_u(t, 0, b);
        for (int k = 0; k < t->C[b].n; ++k) {
            int c = t->C[b].a[k];
            if (!t->box[c].is_leaf) collect_w(t, c, b);
        }
    }
    for (int b = 0; b < t->nbox; ++b)
        for (int k = 0; k < t->W[b].n; ++k) iv_push(&t->X[t->W[b].a[k]], b);
    return t;
}

void or_tree_free(or_tree* t) {
    if (!t) return;
    for (int b = 0; b < t->nbox; ++b) {
        free(t->C[b].a); free(t->U[b].a); free(t->V[b].a); free(t->W[b].a); free(t->X[b].a);
    }
    free(t->C); free(t->U); free(t->V); free(t->W); free(t->X);
    free(t->box); free(t->perm); free(t->qc);
    free(t);
}

int or_tree_nbox(const or_tree* t) { return t ? t->nbox : -1; }

int or_tree_box(const or_tree* t, int b, int64_t* info8) {
    if (!t || b < 0 || b >= t->nbox) return -1;
    const obox* x = &t->box[b];
    info8[0] = x->level;
    info8[1] = x->ijk[0]; info8[2] = x->ijk[1]; info8[3] = x->ijk[2];
    info8[4] = x->parent;
    info8[5] = x->is_leaf;
    info8[6] = x->pbeg;
    info8[7] = x->pend;
    return 0;
}

int or_tree_perm(const or_tree* t, int64_t* perm) {
    if (!t) return -1;
    memcpy(perm, t->perm, sizeof(int64_t) * (size_t)t->n);
    return 0;
}

int or_tree_list(const or_tree* t, int b, int list, int* out, int cap) {
    if (!t || b < 0 || b >= t->nbox || list < 0 || list > 4) return -1;
    const ivec* v = list == 0 ? &t->U[b] : list == 1 ? &t->V[b] : list == 2 ? &t->W[b]
                  : list == 3 ? &t->X[b] : &t->C[b];
    for (int k = 0; k < v->n && k < cap; ++k) out[k] = v->a[k];
    return v->n;
}
