/* tree_internal.h -- oracle octree layout shared by tree.c and fmm.c.
 * TEST INFRASTRUCTURE ONLY (see oracle.h). */
#ifndef DAFMM_ORACLE_TREE_INTERNAL_H
#define DAFMM_ORACLE_TREE_INTERNAL_H
#include <stdint.h>

typedef struct { int n, cap; int* a; } ivec;

typedef struct {
    int level;
    int64_t ijk[3];      /* integer coordinates at this level */
    int parent;
    int child[8];        /* -1 when absent; index c = x | y<<1 | z<<2 */
    int is_leaf;
    int64_t pbeg, pend;  /* particles perm[pbeg..pend) */
} obox;

struct or_tree {
    int64_t n;
    double dom[4];
    int nbox, capbox, maxlev;
    obox* box;
    int64_t* perm;
    int64_t* qc;         /* 21-bit integer coordinates of each particle (input order) */
    ivec *C, *U, *V, *W, *X;
};

int tree_touch(const or_tree* t, int a, int b);
#endif
