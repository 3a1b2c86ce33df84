// Host build of the generated operator code, for checking the generator against the
// oracle without a GPU.  Compiled by tests/test_generator.py with g++.
#include <cmath>
#include <cstdint>

#include "da_common.cuh"
#define DAFMM_INCLUDE_ALL_ORDERS
#include "generated/da_ops_p0.cuh"
#include "generated/da_ops_p1.cuh"
#include "generated/da_ops_p2.cuh"
#include "generated/da_ops_p3.cuh"
#include "generated/da_ops_p4.cuh"
#include "generated/da_ops_p5.cuh"
#include "generated/da_ops_p6.cuh"
#include "generated/da_ops_p7.cuh"
#include "generated/da_ops_p8.cuh"
#include "generated/da_ops_p9.cuh"
#include "generated/da_ops_p10.cuh"
#include "generated/da_tables_p0.h"
#include "generated/da_tables_p1.h"
#include "generated/da_tables_p2.h"
#include "generated/da_tables_p3.h"
#include "generated/da_tables_p4.h"
#include "generated/da_tables_p5.h"
#include "generated/da_tables_p6.h"
#include "generated/da_tables_p7.h"
#include "generated/da_tables_p8.h"
#include "generated/da_tables_p9.h"
#include "generated/da_tables_p10.h"

using namespace dafmm::gen;

template <class T>
struct Store {
    T* o;
    void operator()(int k, T v) const { o[k] = v; }
};
template <class T>
struct Load {
    const T* c;
    T operator()(int k) const { return c[k]; }
};

#define ORDERS(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

template <class T>
static int p2m_any(int p, const T* s, T q, T* out) {
    Store<T> st{out};
    switch (p) {
#define C(P) case P: p2m_o##P<T>(s[0], s[1], s[2], q, st); return 0;
        ORDERS(C)
#undef C
    }
    return -1;
}
// the harmonic-basis P2M: free coefficient j into out[j]
template <class T>
static int p2mh_any(int p, const T* s, T q, T* out) {
    Store<T> st{out};
    switch (p) {
#define C(P) case P: p2mh_o##P<T>(s[0], s[1], s[2], q, st); return 0;
        ORDERS(C)
#undef C
    }
    return -1;
}
template <class T>
static int p2l_any(int p, const T* w, T q, T* out) {
    Store<T> st{out};
    switch (p) {
#define C(P) case P: p2l_o##P<T>(w[0], w[1], w[2], q, st); return 0;
        ORDERS(C)
#undef C
    }
    return -1;
}
template <class T>
static int l2p_any(int p, const T* L, const T* x, T* res4) {
    Load<T> ld{L};
    switch (p) {
#define C(P) case P: l2p_o##P<T>(ld, x[0], x[1], x[2], res4[0], res4[1], res4[2], res4[3]); return 0;
        ORDERS(C)
#undef C
    }
    return -1;
}
template <class T>
static int m2p_any(int p, const T* M, const T* s, T* res4) {
    Load<T> ld{M};
    switch (p) {
#define C(P) case P: m2p_o##P<T>(ld, s[0], s[1], s[2], res4[0], res4[1], res4[2], res4[3]); return 0;
        ORDERS(C)
#undef C
    }
    return -1;
}

extern "C" {
int hc_p2m(int p, int prec, const double* s, double q, double* out, int nc) {
    if (prec == 64) return p2m_any<double>(p, s, q, out);
    float sf[3] = {(float)s[0], (float)s[1], (float)s[2]}, of[300];
    int rc = p2m_any<float>(p, sf, (float)q, of);
    for (int k = 0; k < nc; ++k) out[k] = of[k];
    return rc;
}
int hc_p2mh(int p, int prec, const double* s, double q, double* out, int nh) {
    if (prec == 64) return p2mh_any<double>(p, s, q, out);
    float sf[3] = {(float)s[0], (float)s[1], (float)s[2]}, of[300];
    int rc = p2mh_any<float>(p, sf, (float)q, of);
    for (int k = 0; k < nh; ++k) out[k] = of[k];
    return rc;
}
int hc_p2l(int p, int prec, const double* w, double q, double* out, int nc) {
    if (prec == 64) return p2l_any<double>(p, w, q, out);
    float wf[3] = {(float)w[0], (float)w[1], (float)w[2]}, of[300];
    int rc = p2l_any<float>(p, wf, (float)q, of);
    for (int k = 0; k < nc; ++k) out[k] = of[k];
    return rc;
}
int hc_l2p(int p, int prec, const double* L, const double* x, double* res4, int nc) {
    if (prec == 64) return l2p_any<double>(p, L, x, res4);
    float Lf[300], xf[3] = {(float)x[0], (float)x[1], (float)x[2]}, rf[4];
    for (int k = 0; k < nc; ++k) Lf[k] = (float)L[k];
    int rc = l2p_any<float>(p, Lf, xf, rf);
    for (int k = 0; k < 4; ++k) res4[k] = rf[k];
    return rc;
}
int hc_m2p(int p, int prec, const double* M, const double* s, double* res4, int nc) {
    if (prec == 64) return m2p_any<double>(p, M, s, res4);
    float Mf[300], sf[3] = {(float)s[0], (float)s[1], (float)s[2]}, rf[4];
    for (int k = 0; k < nc; ++k) Mf[k] = (float)M[k];
    int rc = m2p_any<float>(p, Mf, sf, rf);
    for (int k = 0; k < 4; ++k) res4[k] = rf[k];
    return rc;
}
int hc_m2lmap(int p, const double* v, double* inv, double* isq) {
    double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], rho = 1.0 / r2;
    Store<double> a{inv}, b{isq};
    switch (p) {
#define C(P) case P: m2lmap_inv_o##P<double>(v[0], v[1], v[2], rho, a); \
                     m2lmap_isq_o##P<double>(v[0], v[1], v[2], rho, b); return 0;
        ORDERS(C)
#undef C
    }
    return -1;
}
// apply a shift table (0 = M2M, 1 = L2L, 2 = M2M of harmonic multipoles) for octant c: out = T_c in
int hc_shift(int p, int which, int c, const double* in, double* out, int nc) {
    const int* rp = nullptr;
    const unsigned short* col = nullptr;
    const unsigned char* par = nullptr;
    const double* val = nullptr;
    switch (p) {
#define C(P) case P: if (which == 0) { rp = m2m_o##P##_rowptr; col = m2m_o##P##_col; par = m2m_o##P##_par; val = m2m_o##P##_val; } \
                     else if (which == 2) { rp = m2mh_o##P##_rowptr; col = m2mh_o##P##_col; par = m2mh_o##P##_par; val = m2mh_o##P##_val; } \
                     else { rp = l2l_o##P##_rowptr; col = l2l_o##P##_col; par = l2l_o##P##_par; val = l2l_o##P##_val; } break;
        ORDERS(C)
#undef C
        default: return -1;
    }
    for (int b = 0; b < nc; ++b) {
        double s = 0.0;
        for (int k = rp[b]; k < rp[b + 1]; ++k) {
            double v = val[k];
            if (__builtin_popcount(par[k] & c) & 1) v = -v;
            s += v * in[col[k]];
        }
        out[b] = s;
    }
    return 0;
}
}
