// Host-side check of rot_lists.h (the M2L by rotation's structure and task lists), compiled by
// tests/test_rot_lists.py with g++; no GPU.  Returns 0 when every property holds, else the
// number of the first failed property.
#include <algorithm>
#include <cmath>
#include <random>
#include <tuple>
#include <vector>

#include "rot_lists.h"

using namespace dafmm;

namespace {

// the coefficient layout from its definition: all (a, b, c) with a + b + c <= p, ordered by
// degree, then x exponent descending, then y exponent descending
std::vector<std::tuple<int, int, int>> layout(int p) {
    std::vector<std::tuple<int, int, int>> v;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; a + b <= p; ++b)
            for (int c = 0; a + b + c <= p; ++c) v.emplace_back(a, b, c);
    std::sort(v.begin(), v.end(), [](const auto& u, const auto& w) {
        const int nu = std::get<0>(u) + std::get<1>(u) + std::get<2>(u);
        const int nw = std::get<0>(w) + std::get<1>(w) + std::get<2>(w);
        if (nu != nw) return nu < nw;
        if (std::get<0>(u) != std::get<0>(w)) return std::get<0>(u) > std::get<0>(w);
        return std::get<1>(u) > std::get<1>(w);
    });
    return v;
}

double eval(const std::vector<double>& f, const std::vector<std::tuple<int, int, int>>& ex, double x, double y,
            double z) {
    double s = 0.0;
    for (size_t k = 0; k < f.size(); ++k)
        s += f[k] * std::pow(x, std::get<0>(ex[k])) * std::pow(y, std::get<1>(ex[k])) * std::pow(z, std::get<2>(ex[k]));
    return s;
}

// (m+1) x (m+1) matrices of the binary-form substitution p -> al p + be q, q -> ga p + de q,
// packed over m = 0..P: entry [i][j] = coefficient of p^(m-i) q^i in (al p + be q)^(m-j) (ga p + de q)^j
std::vector<double> subst_tables(int P, double al, double be, double ga, double de) {
    std::vector<double> T(rot_off_h(P + 1), 0.0);
    auto binom = [](int n, int k) {
        double r = 1.0;
        for (int t = 0; t < k; ++t) r = r * (n - t) / (t + 1);
        return r;
    };
    for (int m = 0; m <= P; ++m)
        for (int i = 0; i <= m; ++i)
            for (int j = 0; j <= m; ++j) {
                double acc = 0.0;
                for (int k = 0; k <= i; ++k) {
                    if (k > m - j || i - k > j) continue;
                    acc += binom(m - j, k) * binom(j, i - k) * std::pow(al, m - j - k) * std::pow(be, k) *
                           std::pow(ga, j - (i - k)) * std::pow(de, i - k);
                }
                T[rot_off_h(m) + i * (m + 1) + j] = acc;
            }
    return T;
}

// one step as the kernel runs it: every lane walks its tasks in order
std::vector<double> run_step(const std::vector<RotTask>& list, int len, const std::vector<double>& tab,
                             const std::vector<double>& in) {
    std::vector<double> out(in.size() - 1, 0.0);  // in holds nc values and the zero at nc
    for (int lane = 0; lane < 32; ++lane) {
        double s = 0.0;
        for (int t = 0; t < len; ++t) {
            const RotTask w = list[32 * t + lane];
            s += tab[w.x & 0x7fffffffu] * in[w.y & 0xffffu];
            if (w.x >> 31) {
                out[w.y >> 16] = s;
                s = 0.0;
            }
        }
    }
    return out;
}

// every output in exactly one lane, its tasks contiguous with the last flag on the final one,
// expected task counts, padding after the real tasks, lanes balanced; outputs with a zero
// count must not appear (the harmonic lists compute the outputs of z exponent <= 1 only)
int check_list(const RotStructure& r, const std::vector<RotTask>& list, int len, const std::vector<int>& count) {
    const int nc = r.nc;
    if ((int)list.size() != 32 * len) return 1;
    std::vector<int> seen(nc, 0);
    int lmin = len, lmax = 0, biggest = 0;
    for (int k = 0; k < nc; ++k) biggest = std::max(biggest, count[k]);
    for (int lane = 0; lane < 32; ++lane) {
        int t = 0;
        while (t < len && !(list[32 * t + lane].y == (unsigned)nc && list[32 * t + lane].x == 0u)) {
            const int k = (int)(list[32 * t + lane].y >> 16);
            if (k < 0 || k >= nc || seen[k]) return 2;
            seen[k] = 1;
            for (int j = 0; j < count[k]; ++j, ++t) {
                if (t >= len) return 3;
                const RotTask w = list[32 * t + lane];
                if ((int)(w.y >> 16) != k) return 3;
                if ((int)(w.x >> 31) != (j + 1 == count[k] ? 1 : 0)) return 4;
                if ((int)(w.y & 0xffffu) >= nc) return 5;
            }
        }
        lmin = std::min(lmin, t);
        lmax = std::max(lmax, t);
        for (; t < len; ++t)
            if (list[32 * t + lane].y != (unsigned)nc || list[32 * t + lane].x != 0u) return 6;
    }
    for (int k = 0; k < nc; ++k)
        if (seen[k] != (count[k] > 0 ? 1 : 0)) return 7;
    if (lmax != len || lmax - lmin > biggest) return 8;
    return 0;
}

}  // namespace

extern "C" int rot_lists_check(int p, unsigned seed) {
    const RotStructure r = rot_structure(p);
    const auto ex = layout(p);
    const int nc = (int)ex.size();
    // 10: the layout
    if (r.nc != nc) return 10;
    for (int k = 0; k < nc; ++k)
        if (r.ea[k] != std::get<0>(ex[k]) || r.eb[k] != std::get<1>(ex[k]) || r.ec[k] != std::get<2>(ex[k])) return 10;
    // 11: the axial sparsity rule, row by row
    for (int b = 0; b < nc; ++b) {
        std::vector<int> want;
        for (int a = 0; a < nc; ++a) {
            const int db = std::get<1>(ex[b]) - std::get<1>(ex[a]), dc = std::get<2>(ex[b]) - std::get<2>(ex[a]);
            if (db >= 0 && dc >= 0 && db % 2 == 0 && dc % 2 == 0) want.push_back(a);
        }
        if ((int)want.size() != r.rowptr[b + 1] - r.rowptr[b]) return 11;
        for (size_t e = 0; e < want.size(); ++e)
            if (r.col[r.rowptr[b] + e] != want[e]) return 11;
    }
    // 20-22: the three lists
    std::vector<int> cx(nc), cz(nc), ca(nc);
    for (int k = 0; k < nc; ++k) {
        cx[k] = std::get<1>(ex[k]) + std::get<2>(ex[k]) + 1;
        cz[k] = std::get<0>(ex[k]) + std::get<1>(ex[k]) + 1;
        ca[k] = r.rowptr[k + 1] - r.rowptr[k];
    }
    if (int e = check_list(r, r.lx, r.len[0], cx)) return 200 + e;
    if (int e = check_list(r, r.lz, r.len[1], cz)) return 210 + e;
    if (int e = check_list(r, r.la, r.len[2], ca)) return 220 + e;
    // 30, 31: the substitution steps are the substitutions, checked pointwise on random data
    std::mt19937 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (int trial = 0; trial < 3; ++trial) {
        const double al = U(rng), be = U(rng), ga = U(rng), de = U(rng);
        const std::vector<double> T = subst_tables(p, al, be, ga, de);
        std::vector<double> f(nc + 1, 0.0);
        for (int k = 0; k < nc; ++k) f[k] = U(rng);
        const std::vector<double> fx(f.begin(), f.end() - 1);
        const std::vector<double> gx = run_step(r.lx, r.len[0], T, f);  // about x: (y, z) substituted
        const std::vector<double> gz = run_step(r.lz, r.len[1], T, f);  // about z: (x, y) substituted
        for (int pt = 0; pt < 4; ++pt) {
            const double x = 0.6 * U(rng), y = 0.6 * U(rng), z = 0.6 * U(rng);
            const double ref_x = eval(fx, ex, x, al * y + be * z, ga * y + de * z);
            const double ref_z = eval(fx, ex, al * x + be * y, ga * x + de * y, z);
            double scale = 1.0;
            for (double v : fx) scale += std::fabs(v);
            if (std::fabs(eval(gx, ex, x, y, z) - ref_x) > 1e-12 * scale) return 30;
            if (std::fabs(eval(gz, ex, x, y, z) - ref_z) > 1e-12 * scale) return 31;
        }
    }
    return 0;
}

// multiply-adds per pair of the M2L by rotation as the kernel runs it: the real (not padding)
// tasks of the x and z lists, each list run twice, plus those of the axial list
extern "C" long rot_real_tasks(int p) {
    const RotStructure r = rot_structure(p);
    auto real = [&](const std::vector<RotTask>& l) {
        long c = 0;
        for (const RotTask& t : l) c += !(t.y == (unsigned)r.nc && t.x == 0u);
        return c;
    };
    return 2 * real(r.lx) + 2 * real(r.lz) + real(r.la);
}

// The harmonic lists (rot_structure(p, true)): the same checks with only the outputs of z
// exponent c <= 1 present, and, run on random data as the kernel runs them, the same values at
// those outputs as the full lists -- the x-step from a full input, the z-step and the axial step
// from the inputs of z exponent <= 1 alone (the others set to garbage, which must not matter).
extern "C" int rot_lists_check_harm(int p, unsigned seed) {
    const RotStructure r = rot_structure(p);
    const RotStructure h = rot_structure(p, true);
    const auto ex = layout(p);
    const int nc = (int)ex.size();
    if (h.nc != nc || h.rowptr != r.rowptr || h.col != r.col) return 10;
    std::vector<int> cx(nc), cz(nc), ca(nc);
    for (int k = 0; k < nc; ++k) {
        const bool free_k = std::get<2>(ex[k]) <= 1;
        cx[k] = free_k ? std::get<1>(ex[k]) + std::get<2>(ex[k]) + 1 : 0;
        cz[k] = free_k ? std::get<0>(ex[k]) + std::get<1>(ex[k]) + 1 : 0;
        ca[k] = free_k ? r.rowptr[k + 1] - r.rowptr[k] : 0;
    }
    if (int e = check_list(h, h.lx, h.len[0], cx)) return 200 + e;
    if (int e = check_list(h, h.lz, h.len[1], cz)) return 210 + e;
    if (int e = check_list(h, h.la, h.len[2], ca)) return 220 + e;
    std::mt19937 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (int trial = 0; trial < 3; ++trial) {
        const std::vector<double> T = subst_tables(p, U(rng), U(rng), U(rng), U(rng));
        std::vector<double> A(r.col.size());
        for (double& v : A) v = U(rng);
        std::vector<double> f(nc + 1, 0.0), g(nc + 1, 0.0);
        for (int k = 0; k < nc; ++k) {
            f[k] = U(rng);
            g[k] = std::get<2>(ex[k]) <= 1 ? f[k] : 1e30 * U(rng);  // garbage above c = 1
        }
        const std::vector<double> fx = run_step(r.lx, r.len[0], T, f), hx = run_step(h.lx, h.len[0], T, f);
        const std::vector<double> fz = run_step(r.lz, r.len[1], T, f), hz = run_step(h.lz, h.len[1], T, g);
        const std::vector<double> fa = run_step(r.la, r.len[2], A, f), ha = run_step(h.la, h.len[2], A, g);
        for (int k = 0; k < nc; ++k) {
            if (std::get<2>(ex[k]) > 1) continue;
            if (std::fabs(hx[k] - fx[k]) > 1e-12 * (1.0 + std::fabs(fx[k]))) return 30;
            if (std::fabs(hz[k] - fz[k]) > 1e-12 * (1.0 + std::fabs(fz[k]))) return 31;
            if (std::fabs(ha[k] - fa[k]) > 1e-12 * (1.0 + std::fabs(fa[k]))) return 32;
        }
    }
    return 0;
}

// multiply-adds per pair of the harmonic form: its lists' real tasks (x and z lists twice, the
// axial list once) plus two per restored coefficient (one restoration per pair)
extern "C" long rot_real_tasks_harm(int p) {
    const RotStructure r = rot_structure(p, true);
    auto real = [&](const std::vector<RotTask>& l) {
        long c = 0;
        for (const RotTask& t : l) c += !(t.y == (unsigned)r.nc && t.x == 0u);
        return c;
    };
    long restored = 0;
    for (int k = 0; k < r.nc; ++k) restored += r.ec[k] > 1;
    return 2 * real(r.lx) + 2 * real(r.lz) + real(r.la) + 2 * restored;
}
