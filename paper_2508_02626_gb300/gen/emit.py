"""Emit straight-line C++/CUDA for the DA-FMM operators, one set per expansion order.

For every order p this writes ``da_ops_p{p}.cuh`` with

  p2m_o{p}(x, y, z, q, out)       P2M of one charge (Eq. 2) in scaled offsets
  p2mh_o{p}(x, y, z, q, out)      the same, free coefficients of the harmonic basis only
  p2l_o{p}(X, Y, Z, q, out)       P2L of one charge (Eq. 6), w = centre - source, scaled
  l2p_o{p}(L, x, y, z, ...)       L2P with gradient (Sec. 3.2)
  m2p_o{p}(M, x, y, z, ...)       M2P with gradient (Sec. 3.2)
  m2lmap_o{p}(X, Y, Z, inv, isq)  the M2L transfer-map factors (Eq. 5)

and ``da_tables_p{p}.h`` with the level-independent M2M (Eq. 4, octant-reduced
as in Sec. 3.3, also in the harmonic basis) and L2L (Eq. 7) matrices in compressed rows.

Like the paper's parser, the emitter walks the symbolic coefficients term by
term (sign, rational coefficient, powers of the base symbols), computes every
distinct power product once (each as one multiplication of an already
computed product) and emits each coefficient as a sum of rational multiples
of those products.  The code is ``__host__ __device__`` so that a host build
can be checked against the oracle without a GPU.
"""
import argparse
import os
import sys
from fractions import Fraction

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
    from paper_2508_02626_gb300.gen import operators as ops  # noqa: E402
    from paper_2508_02626_gb300.gen.sda import exponents, index, ncoef  # noqa: E402
else:
    from . import operators as ops
    from .sda import exponents, index, ncoef

MAXORD = 10


def lit(fr):
    """A rational as a C double literal (17 significant digits)."""
    fr = Fraction(fr)
    if fr.denominator == 1 and abs(fr.numerator) < 2 ** 53:
        return "%d.0" % fr.numerator
    return "%.17g" % (fr.numerator / fr.denominator)


class MonoPlan:
    """Power products of the base symbols, each built from an earlier one by one product.

    Products are emitted lazily, right before the first output that needs them, so that
    the live set stays close to what the current output order uses."""

    def __init__(self, syms, base_name, base_expr):
        self.syms = syms
        self.zero = (0,) * len(syms)
        self.name = {self.zero: base_name}
        self.lines = ["const T %s = %s;" % (base_name, base_expr)]
        self.count = 0

    def get(self, e):
        """Name of the product e, emitting it (and missing factors) when needed."""
        if e in self.name:
            return self.name[e]
        # prefer a factor that already exists
        k_best = None
        for k in range(len(e)):
            if e[k] > 0 and (e[:k] + (e[k] - 1,) + e[k + 1:]) in self.name:
                k_best = k
                break
        if k_best is None:
            k_best = next(k for k in range(len(e)) if e[k] > 0)
        pe = e[:k_best] + (e[k_best] - 1,) + e[k_best + 1:]
        pn = self.get(pe)
        nm = "m%d" % self.count
        self.count += 1
        self.lines.append("const T %s = %s * %s;" % (nm, pn, self.syms[k_best]))
        self.name[e] = nm
        return nm


def sum_expr(terms, nacc=1):
    """terms: list of (Fraction coefficient, operand name).  Returns a C expression."""
    parts = []
    for c, nm in terms:
        if c == 1:
            parts.append("+ %s" % nm)
        elif c == -1:
            parts.append("- %s" % nm)
        elif c > 0:
            parts.append("+ T(%s) * %s" % (lit(c), nm))
        else:
            parts.append("- T(%s) * %s" % (lit(-c), nm))
    if not parts:
        return "T(0)"
    s = " ".join(parts)
    if s.startswith("+ "):
        s = s[2:]
    return s


def emit_poly_outputs(name, p, syms, coefs, base_name, base_expr, args, pre_lines, out_scale=None):
    plan = MonoPlan(syms, base_name, base_expr)
    nterm = 0
    for k, poly in enumerate(coefs):
        terms = [(c, plan.get(e)) for e, c in sorted(poly.t.items(), key=lambda kv: (sum(kv[0]), kv[0]))]
        nterm += len(terms)
        plan.lines.append("out(%d, %s);" % (k, sum_expr(terms)))
    body = list(pre_lines) + plan.lines
    head = "template <class T, class Out>\nDAFMM_HD DAFMM_INLINE void %s(%s, Out&& out) {\n" % (name, args)
    return head + "".join("    %s\n" % l for l in body) + "}\n", plan.count + nterm


def emit_eval(name, p, kind):
    """L2P (kind='l2p') or M2P (kind='m2p') with gradient.  For each (a, b) the column
    sum_c C[a,b,c] z^c and its z-derivative are formed by Horner's rule, then weighted by
    x^a y^b (and a x^(a-1) y^b, b x^a y^(b-1) for the x and y derivatives)."""
    lines = []
    args = "const Src& C, T x, T y, T z, T& phi, T& gx, T& gy, T& gz"
    if kind == "l2p":
        lines.append("const T u0 = x, u1 = y, u2 = z;")
    else:
        lines += ["const T R2 = x * x + y * y + z * z;",
                  "const T rho = dafmm_rcp(R2);",
                  "const T nd = dafmm_sqrt(rho);",
                  "const T u0 = x * rho, u1 = y * rho, u2 = z * rho;"]
    lines += ["T F = T(0), G0 = T(0), G1 = T(0), G2 = T(0);"]
    # powers of u0 and u1 up to p
    for k in range(2, p + 1):
        lines.append("const T xa%d = %s * u0;" % (k, "u0" if k == 2 else "xa%d" % (k - 1)))
    xa = lambda k: "T(1)" if k == 0 else ("u0" if k == 1 else "xa%d" % k)
    for a in range(p + 1):
        lines.append("{")
        # y^b x^a built incrementally inside the column loop
        for b in range(p - a + 1):
            cmax = p - a - b
            # Horner: H = sum_c C[a,b,c] z^c, D = dH/dz
            cidx = [index(a, b, c) for c in range(cmax + 1)]
            hl = ["T H = C(%d);" % cidx[cmax]]
            if cmax >= 1:
                hl.append("T D = T(0);")
                for c in range(cmax - 1, -1, -1):
                    hl.append("D = dafmm_fma(D, u2, H);")
                    hl.append("H = dafmm_fma(H, u2, C(%d));" % cidx[c])
            else:
                hl.append("const T D = T(0);")
            # weights: yb = x^a y^b, ybm = x^a y^(b-1), xbm = x^(a-1) y^b
            if b == 0:
                lines.append("T yb = %s;" % xa(a))
                lines.append("T ybm = T(0);")
                lines.append("T xbm = %s;" % (xa(a - 1) if a >= 1 else "T(0)"))
            else:
                lines.append("ybm = yb;")
                lines.append("yb = yb * u1;")
                if a >= 1:
                    lines.append("xbm = xbm * u1;")
            lines.append("{")
            lines += ["  " + h for h in hl]
            lines.append("  F = dafmm_fma(yb, H, F);")
            lines.append("  G2 = dafmm_fma(yb, D, G2);")
            if a >= 1:
                lines.append("  G0 = dafmm_fma(T(%d) * xbm, H, G0);" % a)
            if b >= 1:
                lines.append("  G1 = dafmm_fma(T(%d) * ybm, H, G1);" % b)
            lines.append("}")
        lines.append("}")
    if kind == "l2p":
        lines += ["phi = F;", "gx = G0;", "gy = G1;", "gz = G2;"]
    else:
        lines += ["phi = nd * F;",
                  "const T fr = F * nd * R2;  /* phi_M / |d|, since 1/|d| = |s| = sqrt(R2) */",
                  "const T a0 = u0 * fr + nd * G0, a1 = u1 * fr + nd * G1, a2 = u2 * fr + nd * G2;",
                  "const T sa = x * a0 + y * a1 + z * a2;",
                  "const T tw = T(2) * rho * rho * sa;",
                  "gx = rho * a0 - tw * x;",
                  "gy = rho * a1 - tw * y;",
                  "gz = rho * a2 - tw * z;"]
    head = "template <class T, class Src>\nDAFMM_HD DAFMM_INLINE void %s(%s) {\n" % (name, args)
    return head + "".join("    %s\n" % l for l in lines) + "}\n"


def csr_table(name, p, table, with_parity=True):
    ex = exponents(p)
    nc = ncoef(p)
    # within a row, entries are ordered by parity pattern, then column: the shift kernels sum
    # each parity class separately (a Hadamard transform over the 8 octants does the rest)
    rowptr, cols, vals, par = [0], [], [], []
    for b in range(nc):
        row = []
        for a in range(nc):
            v = table[b][a]
            if v:
                m = 0
                for k in range(3):
                    if (ex[b][k] + ex[a][k]) % 2:
                        m |= 1 << k
                row.append((m, a, v))
        for m, a, v in sorted(row, key=lambda t: (t[0], t[1])):
            cols.append(a)
            vals.append(v)
            par.append(m)
        rowptr.append(len(cols))
    out = []
    out.append("static const int %s_nnz = %d;\n" % (name, len(cols)))
    out.append("static const int %s_rowptr[%d] = {%s};\n" % (name, nc + 1, ",".join(map(str, rowptr))))
    out.append("static const unsigned short %s_col[%d] = {%s};\n" % (name, max(1, len(cols)),
                                                                   ",".join(map(str, cols)) or "0"))
    out.append("static const unsigned char %s_par[%d] = {%s};\n" % (name, max(1, len(par)),
                                                                  ",".join(map(str, par)) or "0"))
    vl = []
    for i, v in enumerate(vals):
        vl.append(lit(v))
    out.append("static const double %s_val[%d] = {\n%s};\n" % (name, max(1, len(vals)),
                                                            ",\n".join(",".join(vl[i:i + 6]) for i in range(0, len(vl), 6)) or "0"))
    return "".join(out), len(cols)


HEADER = """// GENERATED by paper_2508_02626_gb300/gen/emit.py -- do not edit.
// Straight-line DA-FMM operators of expansion order %(p)d (%(nc)d coefficients),
// derived by symbolic DA from the paper's Eqs. 2, 5 and 6 and the evaluation of Sec. 3.2.
"""


def generate(p, outdir):
    nc = ncoef(p)
    parts = [HEADER % dict(p=p, nc=nc)]
    parts.append("#pragma once\n#include \"../da_common.cuh\"\nnamespace dafmm {\nnamespace gen {\n\n")
    stats = {}
    syms, c = ops.p2m(p)
    code, n = emit_poly_outputs(
        "p2m_o%d" % p, p, ("x", "y", "z", "R2"), c, "qq", "q", "T x, T y, T z, T q",
        ["const T R2 = x * x + y * y + z * z;"])
    parts.append("// P2M, Eq. 2: out(k, q * coefficient k of (1 - 2 s.d + s^2 d^2)^(-1/2)), s = (x,y,z)\n")
    parts.append(code + "\n")
    stats["p2m"] = n
    free = ops.free_coefficients(p)
    code, n = emit_poly_outputs(
        "p2mh_o%d" % p, p, ("x", "y", "z", "R2"), [c[i] for i in free], "qq", "q", "T x, T y, T z, T q",
        ["const T R2 = x * x + y * y + z * z;"])
    parts.append("// P2M in the harmonic basis: out(j, coefficient of free index j), the (p + 1)^2 coefficients\n"
                 "// of z exponent <= 1 in layout order (the others follow by Laplace's equation)\n")
    parts.append(code + "\n")
    stats["p2mh"] = n
    syms, c = ops.p2l(p)
    code, n = emit_poly_outputs(
        "p2l_o%d" % p, p, ("X", "Y", "Z", "rho"), c, "qir", "q * ir", "T X, T Y, T Z, T q",
        ["const T R2 = X * X + Y * Y + Z * Z;", "const T ir = dafmm_rsqrt(R2);", "const T rho = ir * ir;"])
    parts.append("// P2L, Eq. 6: out(k, q * coefficient k of 1/|w + d'|), w = (X,Y,Z)\n")
    parts.append(code + "\n")
    stats["p2l"] = n
    parts.append("// L2P: phi = L(x), g = grad L(x) (Sec. 3.2)\n")
    parts.append(emit_eval("l2p_o%d" % p, p, "l2p") + "\n")
    parts.append("// M2P: phi = |d| M(d), d = s/|s|^2, g = grad_s phi (Sec. 3.2)\n")
    parts.append(emit_eval("m2p_o%d" % p, p, "m2p") + "\n")
    syms, inv, isq = ops.m2l_map(p)
    code1, n1 = emit_poly_outputs(
        "m2lmap_inv_o%d" % p, p, ("X", "Y", "Z", "rho"), inv, "one", "T(1)", "T X, T Y, T Z, T rho", [])
    code2, n2 = emit_poly_outputs(
        "m2lmap_isq_o%d" % p, p, ("X", "Y", "Z", "rho"), isq, "one", "T(1)", "T X, T Y, T Z, T rho", [])
    parts.append("// M2L map, Eq. 5: |v+u|^2 = |v|^2 (1+t), t = rho (2 v.u + u.u), rho = 1/|v|^2;\n"
                 "// m2lmap_inv: coefficients of (1+t)^-1, m2lmap_isq: of (1+t)^-1/2\n")
    parts.append(code1 + "\n" + code2 + "\n")
    stats["m2lmap"] = n1 + n2
    parts.append("}  // namespace gen\n}  // namespace dafmm\n")
    with open(os.path.join(outdir, "da_ops_p%d.cuh" % p), "w") as f:
        f.write("".join(parts))

    tparts = [HEADER % dict(p=p, nc=nc), "#pragma once\nnamespace dafmm {\nnamespace gen {\n\n"]
    tparts.append("// M2M (Eq. 4) in scaled variables, child octant (0,0,0): M~'_b = sum T[b][a] M~_a.\n"
                  "// Octant c flips the sign of entry (b,a) when popcount(par & c) is odd (Sec. 3.3).\n")
    T = ops.m2m_scaled_table(p)
    code, nnz = csr_table("m2m_o%d" % p, p, T)
    tparts.append(code)
    stats["m2m_nnz"] = nnz
    tparts.append("\n// M2M of harmonic multipoles: the free rows of the table above composed with the expansion\n"
                  "// from the free coefficients (Laplace's equation); reads and writes free coefficients only.\n")
    code, nnz = csr_table("m2mh_o%d" % p, p, ops.m2m_harmonic_table(p, T))
    tparts.append(code)
    stats["m2mh_nnz"] = nnz
    tparts.append("\n// L2L (Eq. 7) in scaled variables, child octant (0,0,0): L~'_b = sum T[b][a] L~_a.\n")
    code, nnz = csr_table("l2l_o%d" % p, p, ops.l2l_scaled_table(p))
    tparts.append(code)
    stats["l2l_nnz"] = nnz
    tparts.append("\n}  // namespace gen\n}  // namespace dafmm\n")
    with open(os.path.join(outdir, "da_tables_p%d.h" % p), "w") as f:
        f.write("".join(tparts))
    return stats


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--orders", default="0-%d" % MAXORD)
    a = ap.parse_args(argv)
    lo, hi = (int(x) for x in a.orders.split("-")) if "-" in a.orders else (int(a.orders),) * 2
    os.makedirs(a.out, exist_ok=True)
    for p in range(lo, hi + 1):
        st = generate(p, a.out)
        print("order %d: %s" % (p, st))


if __name__ == "__main__":
    main()
