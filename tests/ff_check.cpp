// Host check of the float-float arithmetic (csrc/ff.cuh) against long double: random operands
// over a range of magnitudes and signs (cancelling sums included), relative errors of add, mul,
// rsqrt and rcp; and the generated P2M and L2P of orders 2..10 evaluated in float-float against
// FP64.  Prints the largest relative errors as "name value" lines.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <random>

#include "ff.cuh"
#include "generated/da_ops_p2.cuh"
#include "generated/da_ops_p3.cuh"
#include "generated/da_ops_p4.cuh"
#include "generated/da_ops_p5.cuh"
#include "generated/da_ops_p6.cuh"
#include "generated/da_ops_p7.cuh"
#include "generated/da_ops_p8.cuh"
#include "generated/da_ops_p9.cuh"
#include "generated/da_ops_p10.cuh"

using dafmm::ff;
using namespace dafmm::gen;

#define ORDERS(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

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
template <class T>
static void p2m_any(int p, T x, T y, T z, T q, T* out) {
    Store<T> st{out};
    switch (p) {
#define C(P) case P: p2m_o##P<T>(x, y, z, q, st); return;
        ORDERS(C)
#undef C
    }
}
template <class T>
static void l2p_any(int p, const T* c, T x, T y, T z, T* out4) {
    Load<T> ld{c};
    switch (p) {
#define C(P) case P: l2p_o##P<T>(ld, x, y, z, out4[0], out4[1], out4[2], out4[3]); return;
        ORDERS(C)
#undef C
    }
}

static long double ld(ff a) { return (long double)a.hi + (long double)a.lo; }
static ff from_ld(long double x) {
    const float h = (float)x;
    return ff(h, (float)(x - (long double)h));
}

int main() {
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<double> U(-1.0, 1.0), E(-20.0, 20.0);
    double e_add = 0, e_mul = 0, e_rsq = 0, e_rcp = 0, e_canc = 0;
    for (int i = 0; i < 200000; ++i) {
        const long double x = (long double)U(rng) * powl(2.0L, (long double)(int)E(rng));
        const long double y = (long double)U(rng) * powl(2.0L, (long double)(int)E(rng));
        const ff a = from_ld(x), b = from_ld(y);
        const long double xa = ld(a), yb = ld(b);
        const long double s = xa + yb, p = xa * yb;
        if (s != 0) e_add = fmax(e_add, (double)fabsl((ld(dafmm::ff_add(a, b)) - s) / s));
        if (p != 0) e_mul = fmax(e_mul, (double)fabsl((ld(dafmm::ff_mul(a, b)) - p) / p));
        const long double ax = fabsl(xa);
        if (ax > 0) {
            const ff aa(a.hi < 0 ? -a.hi : a.hi, a.hi < 0 ? -a.lo : a.lo);
            e_rsq = fmax(e_rsq, (double)fabsl((ld(dafmm::ff_rsqrt(aa)) - 1.0L / sqrtl(ax)) * sqrtl(ax)));
            e_rcp = fmax(e_rcp, (double)fabsl((ld(dafmm::ff_rcp(a)) - 1.0L / xa) * xa));
        }
        // nearly cancelling sums: the error bound is relative to the result as well
        const ff c = from_ld(-xa * (1.0L + 1e-6L * (long double)U(rng)));
        const long double sc = xa + ld(c);
        if (sc != 0) e_canc = fmax(e_canc, (double)fabsl((ld(dafmm::ff_add(a, c)) - sc) / sc));
    }
    printf("add %.3e\nmul %.3e\nrsqrt %.3e\nrcp %.3e\ncancel %.3e\n", e_add, e_mul, e_rsq, e_rcp, e_canc);
    // generated operators in float-float against FP64 (relative to the largest coefficient)
    double e_p2m = 0, e_l2p = 0;
    std::uniform_real_distribution<double> S(-0.5, 0.5);
    for (int p = 2; p <= 10; ++p) {
        const int nc = (p + 1) * (p + 2) * (p + 3) / 6;
        for (int it = 0; it < 200; ++it) {
            const double x = S(rng), y = S(rng), z = S(rng), q = U(rng);
            double c64[286];
            ff cffv[286];
            p2m_any<double>(p, x, y, z, q, c64);
            p2m_any<ff>(p, ff(x), ff(y), ff(z), ff(q), cffv);
            double mx = 0, d = 0;
            for (int k = 0; k < nc; ++k) {
                mx = fmax(mx, fabs(c64[k]));
                d = fmax(d, fabs(cffv[k].to_double() - c64[k]));
            }
            e_p2m = fmax(e_p2m, d / mx);
            double o64[4];
            ff off[4];
            l2p_any<double>(p, c64, x, y, z, o64);
            ff cf[286];
            for (int k = 0; k < nc; ++k) cf[k] = ff(c64[k]);
            l2p_any<ff>(p, cf, ff(x), ff(y), ff(z), off);
            const double F64 = o64[0];
            const double g64[3] = {o64[1], o64[2], o64[3]};
            const ff Fff = off[0];
            const ff gff[3] = {off[1], off[2], off[3]};
            double sc = 0;
            for (int k = 0; k < nc; ++k) sc += fabs(c64[k]);
            e_l2p = fmax(e_l2p, fabs(Fff.to_double() - F64) / sc);
            for (int v = 0; v < 3; ++v) e_l2p = fmax(e_l2p, fabs(gff[v].to_double() - g64[v]) / (sc * p));
        }
    }
    printf("gen_p2m %.3e\ngen_l2p %.3e\n", e_p2m, e_l2p);
    return 0;
}
