// rot_lists.h -- host-side structure of the M2L by rotation (Sec. 3.4), plain C++ (no CUDA).
//
// For order p (nc coefficients in the layout: degree graded, x exponent descending, then y):
//   * the structural non-zeros of the axial M2L matrix A_rho (displacement (rho, 0, 0)), CSR by
//     output row: column (a, b, c) reaches row (a', b', c') only when b' >= b, c' >= c and both
//     differences are even -- the axial transfer map sees y and z only through y^2 + z^2 and
//     odd powers of y and z;
//   * the kernel's task lists of the five steps.  A step computes out[k] = sum of its tasks
//     tab[offset] * in[index]:
//       x-step (substitution about x): output (a, b, c) takes the binary form of degree
//         m = b + c at fixed x exponent a, row c of the (m+1) x (m+1) substitution matrix;
//       z-step (about z): output (a, b, c) takes the form of degree m = a + b at fixed z
//         exponent c, row b;
//       axial step: output row b takes the CSR entries of row b.
//     The outputs are dealt to 32 lanes, largest first, each onto the least loaded lane; a
//     lane's tasks run in order, whole outputs at a time, and every lane's list is padded to
//     the longest with tasks that read index nc (a zero the kernel keeps there).  Task t of
//     lane l is list[32 t + l]: x = offset | last-task-of-its-output << 31,
//     y = input index | output index << 16.
// Substitution matrices are packed per degree m at offset rot_off(m) = sum_{m' < m} (m'+1)^2.
// With harm, the lists compute only the outputs of z exponent c <= 1 -- the free coefficients of
// a harmonic expansion (every vector of the M2L is one): a z-step output and an axial output of
// z exponent c <= 1 read only inputs of z exponent <= c, so from the x-step on the free
// coefficients carry the computation; the kernel restores the others (Laplace's equation) before
// the last x-step, whose inputs span every z exponent, and once per target at the end.
#pragma once
#include <algorithm>
#include <vector>

namespace dafmm {

struct RotTask {
    unsigned x, y;
};

struct RotStructure {
    int nc = 0;
    std::vector<int> ea, eb, ec;       // exponents of each coefficient
    std::vector<int> rowptr;           // axial CSR (nc + 1)
    std::vector<unsigned short> col;
    std::vector<RotTask> lx, lz, la;   // [len][32] each
    int len[3] = {0, 0, 0};            // x-step, z-step, axial
};

inline int rot_deg_start(int n) { return n * (n + 1) * (n + 2) / 6; }
inline int rot_coef_index(int n, int a, int c) { return rot_deg_start(n) + (n - a) * (n - a + 1) / 2 + c; }
inline int rot_off_h(int m) { return m * (m + 1) * (2 * m + 1) / 6; }

inline RotStructure rot_structure(int p, bool harm = false) {
    RotStructure r;
    for (int n = 0; n <= p; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                r.ea.push_back(a);
                r.eb.push_back(b);
                r.ec.push_back(n - a - b);
            }
    const int nc = r.nc = (int)r.ea.size();
    r.rowptr.assign(1, 0);
    for (int b = 0; b < nc; ++b) {
        for (int a = 0; a < nc; ++a)
            if (r.eb[b] >= r.eb[a] && r.ec[b] >= r.ec[a] && (r.eb[b] - r.eb[a]) % 2 == 0 &&
                (r.ec[b] - r.ec[a]) % 2 == 0)
                r.col.push_back((unsigned short)a);
        r.rowptr.push_back((int)r.col.size());
    }
    struct Task {
        unsigned off, in;
    };
    auto build = [&](const std::vector<std::vector<Task>>& per_out, std::vector<RotTask>& list) {
        std::vector<int> order(nc);
        for (int k = 0; k < nc; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](int u, int v) { return per_out[u].size() > per_out[v].size(); });
        std::vector<std::vector<RotTask>> lane(32);
        for (int k : order) {
            int best = 0;
            for (int q = 1; q < 32; ++q)
                if (lane[q].size() < lane[best].size()) best = q;
            for (size_t j = 0; j < per_out[k].size(); ++j) {
                const bool last = j + 1 == per_out[k].size();
                lane[best].push_back(
                    RotTask{per_out[k][j].off | (last ? 0x80000000u : 0u), per_out[k][j].in | ((unsigned)k << 16)});
            }
        }
        size_t len = 0;
        for (auto& v : lane) len = std::max(len, v.size());
        list.assign(len * 32, RotTask{0u, (unsigned)nc});
        for (int q = 0; q < 32; ++q)
            for (size_t t = 0; t < lane[q].size(); ++t) list[t * 32 + q] = lane[q][t];
        return (int)len;
    };
    std::vector<std::vector<Task>> tx(nc), tz(nc), ta(nc);
    for (int k = 0; k < nc; ++k) {
        const int a = r.ea[k], b = r.eb[k], c = r.ec[k], n = a + b + c;
        if (harm && c > 1) continue;
        const int mx = b + c, mz = a + b;
        for (int j = 0; j <= mx; ++j)
            tx[k].push_back({(unsigned)(rot_off_h(mx) + c * (mx + 1) + j), (unsigned)(rot_coef_index(n, a, 0) + j)});
        for (int j = 0; j <= mz; ++j)
            tz[k].push_back({(unsigned)(rot_off_h(mz) + b * (mz + 1) + j), (unsigned)rot_coef_index(n, mz - j, c)});
        for (int e = r.rowptr[k]; e < r.rowptr[k + 1]; ++e) ta[k].push_back({(unsigned)e, (unsigned)r.col[e]});
    }
    r.len[0] = build(tx, r.lx);
    r.len[1] = build(tz, r.lz);
    r.len[2] = build(ta, r.la);
    return r;
}

}  // namespace dafmm
