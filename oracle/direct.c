/*
 * direct.c -- the pairwise Coulomb sum of Eq. 1 (the "analytical solution"
 * the paper's error sigma is measured against, Sec. 3.5), plus the small
 * pthreads parallel-for the oracle uses.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include "oracle_internal.h"

typedef struct {
    int64_t n, nchunk, next;
    pfor_fn fn;
    void* arg;
} pfor_job;

static void* pfor_thread(void* p) {
    pfor_job* j = (pfor_job*)p;
    for (;;) {
        int64_t c = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (c >= j->nchunk) break;
        j->fn(j->n * c / j->nchunk, j->n * (c + 1) / j->nchunk, j->arg);
    }
    return NULL;
}

void parallel_for(int64_t n, int nthreads, pfor_fn fn, void* arg) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n <= 0) return;
    if (nthreads == 1 || n < 2) {
        fn(0, n, arg);
        return;
    }
    /* chunks handed out from a shared counter */
    pfor_job job = {n, (int64_t)nthreads * 16, 0, fn, arg};
    if (job.nchunk > n) job.nchunk = n;
    pthread_t th[256];
    for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, pfor_thread, &job);
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
}

/* Neumaier's improvement of Kahan summation */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

typedef struct {
    int64_t n;
    const double *xyz, *q;
    const int64_t* tgt;
    double *phi, *field;
} direct_arg;

static void direct_range(int64_t b, int64_t e, void* p) {
    direct_arg* a = (direct_arg*)p;
    for (int64_t k = b; k < e; ++k) {
        int64_t i = a->tgt ? a->tgt[k] : k;
        const double* ri = a->xyz + 3 * i;
        nsum ph = {0, 0}, f[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int64_t j = 0; j < a->n; ++j) {
            if (j == i) continue;
            double dx = ri[0] - a->xyz[3 * j], dy = ri[1] - a->xyz[3 * j + 1], dz = ri[2] - a->xyz[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue; /* coincident points contribute nothing */
            double r = sqrt(r2);
            double qr = a->q[j] / r;
            nadd(&ph, qr);
            double qr3 = qr / r2;
            nadd(&f[0], qr3 * dx);
            nadd(&f[1], qr3 * dy);
            nadd(&f[2], qr3 * dz);
        }
        a->phi[k] = ph.s + ph.c;
        for (int c = 0; c < 3; ++c) a->field[3 * k + c] = f[c].s + f[c].c;
    }
}

int or_direct(int64_t n, const double* xyz, const double* q, int64_t nt, const int64_t* tgt,
              double* phi, double* field, int nthreads) {
    if (n < 0) return -1;
    if (!tgt) nt = n;
    for (int64_t k = 0; tgt && k < nt; ++k)
        if (tgt[k] < 0 || tgt[k] >= n) return -1;
    direct_arg a = {n, xyz, q, tgt, phi, field};
    parallel_for(nt, nthreads, direct_range, &a);
    return 0;
}
