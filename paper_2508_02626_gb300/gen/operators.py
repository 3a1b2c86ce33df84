"""Symbolic-DA derivations of the DA-FMM operators (paper Sec. 2 and 3).

Each function runs the operator's DA algorithm on symbols and returns the
explicit coefficient expressions; ``emit.py`` turns them into straight-line
CUDA.  Everything is in box-scaled variables (a box of width h becomes a box
of width 1), which makes every table independent of the tree level:

  multipole   M~_a = M_a / h^|a|     (P2M of s equals P2M of s/h, Eq. 2 is homogeneous)
  local       L~_b = L_b h^|b|       (then L~ = (1/h) K^ M~ for M2L, Eq. 5)
"""
from fractions import Fraction

from .sda import SDA, Poly, exponents, index, ncoef


# ---- P2M, Eq. 2 -------------------------------------------------------------------------
def p2m(p):
    """Coefficients of (1 - 2 s.d + s^2 d^2)^(-1/2) as polynomials in x, y, z, R2 = s.s.
    The constant part of v is exactly 1, so the series needs no substitution; s^2 is
    carried as the symbol R2 (the paper's r substitution)."""
    syms = ("x", "y", "z", "R2")
    w = SDA(p, syms)
    if p >= 1:
        for k, s in enumerate(("x", "y", "z")):
            w.c[index(int(k == 0), int(k == 1), int(k == 2))] = Poly.sym(syms, s, 1, -2)
    if p >= 2:
        for k in range(3):
            w.c[index(2 * (k == 0), 2 * (k == 1), 2 * (k == 2))] = Poly.sym(syms, "R2")
    res = w.pow_unit(Fraction(-1, 2))
    return syms, res.c


# ---- P2L, Eq. 6 -------------------------------------------------------------------------
def p2l(p):
    """Coefficients of 1/|w + d'| about w = (X, Y, Z): v = |w|^2 (1 + t) with
    t = rho (2 w.d' + d'.d'), rho = 1/|w|^2 (the constant part reset to a symbol);
    the result is |w|^-1 times the returned polynomials in X, Y, Z, rho."""
    syms = ("X", "Y", "Z", "rho")
    t = SDA(p, syms)
    if p >= 1:
        for k, s in enumerate(("X", "Y", "Z")):
            e = [0, 0, 0, 0]
            e[k] = 1
            e[3] = 1
            t.c[index(int(k == 0), int(k == 1), int(k == 2))] = Poly(syms, {tuple(e): Fraction(2)})
    if p >= 2:
        for k in range(3):
            t.c[index(2 * (k == 0), 2 * (k == 1), 2 * (k == 2))] = Poly.sym(syms, "rho")
    res = t.pow_unit(Fraction(-1, 2))
    return syms, res.c


# ---- M2L transfer map, Eq. 5 -------------------------------------------------------------
def m2l_map(p):
    """The pieces of M2: R = 1/|v + u|^2 and sqrt(R), with v = (X, Y, Z) the box
    displacement.  |v+u|^2 = |v|^2 (1 + t), t = rho (2 v.u + u.u); R = rho (1+t)^-1,
    sqrt(R) = sqrt(rho) (1+t)^-1/2.  Returns polynomials in X, Y, Z, rho for
    (1+t)^-1 and (1+t)^-1/2."""
    syms = ("X", "Y", "Z", "rho")
    t = SDA(p, syms)
    if p >= 1:
        for k, s in enumerate(("X", "Y", "Z")):
            e = [0, 0, 0, 0]
            e[k] = 1
            e[3] = 1
            t.c[index(int(k == 0), int(k == 1), int(k == 2))] = Poly(syms, {tuple(e): Fraction(2)})
    if p >= 2:
        for k in range(3):
            t.c[index(2 * (k == 0), 2 * (k == 1), 2 * (k == 2))] = Poly.sym(syms, "rho")
    inv = t.pow_unit(-1)
    isq = t.pow_unit(Fraction(-1, 2))
    return syms, inv.c, isq.c


# ---- M2M, Eq. 3-4, with the octant reduction of Sec. 3.3 ----------------------------------
def m2m_matrix(p, signs=(1, 1, 1)):
    """Symbolic M2M for r0 = (s1 a, s2 a, s3 a): the map M1 depends on the single
    scalar a (Sec. 3.3).  Returns T[beta][alpha] as polynomials in a, with
    M'_beta = sum_alpha T[beta][alpha] M_alpha."""
    syms = ("a",)
    A = Poly.sym(syms, "a")
    one = Poly.const(syms, 1)
    dd = SDA(p, syms)
    if p >= 2:
        for k in range(3):
            dd.c[index(2 * (k == 0), 2 * (k == 1), 2 * (k == 2))] = one
    # 1 + r0^2 d'^2 + 2 r0.d'  =  1 + t
    t = dd.scale_poly(A * A * Poly.const(syms, 3))
    if p >= 1:
        for k in range(3):
            t.c[index(int(k == 0), int(k == 1), int(k == 2))] = A.scale(2 * signs[k])
    R = t.pow_unit(-1)
    sR = t.pow_unit(Fraction(-1, 2))
    maps = []
    for k in range(3):
        dv = SDA.var(p, syms, k)
        maps.append((dv + dd.scale_poly(A.scale(signs[k]))) * R)
    # columns: sqrt(R) * M1^alpha
    ex = exponents(p)
    nc = ncoef(p)
    mono = [None] * nc
    mono[0] = SDA.const(p, syms, one)
    cols = [None] * nc
    for i in range(nc):
        e = list(ex[i])
        if i > 0:
            v = 0 if e[0] else (1 if e[1] else 2)
            e[v] -= 1
            mono[i] = mono[index(*e)] * maps[v]
        cols[i] = sR * mono[i]
    return [[cols[a].c[b] for a in range(nc)] for b in range(nc)]


def m2m_scaled_table(p):
    """Level-independent M2M for the (+,+,+) octant in scaled variables: child width 1,
    r0 = (1/2, 1/2, 1/2), parent coefficients scaled by (parent width)^-|beta| = 2^-|beta|.
    Returns a dense nc x nc list of Fractions (row beta, column alpha)."""
    T = m2m_matrix(p, (1, 1, 1))
    ex = exponents(p)
    nc = ncoef(p)
    out = [[Fraction(0)] * nc for _ in range(nc)]
    for b in range(nc):
        nb = sum(ex[b])
        for a in range(nc):
            val = T[b][a].subs_number("a", Fraction(1, 2)).as_number()
            out[b][a] = val / (2 ** nb)
    return out


def l2l_scaled_table(p):
    """Level-independent L2L (Eq. 7) for the child in octant (0,0,0) in scaled variables:
    parent width 1, r0 = child centre - parent centre = (-1/4, -1/4, -1/4), child
    coefficients scaled by (1/2)^|beta|.
    L'_beta = sum_{alpha >= beta} C(alpha, beta) r0^(alpha-beta) L_alpha (the composition with the
    linear shift M3, done symbolically in r0 = (x0, y0, z0) and then evaluated)."""
    syms = ("x0", "y0", "z0")
    maps = [SDA.var(p, syms, k, Poly.sym(syms, s)) for k, s in enumerate(syms)]
    ex = exponents(p)
    nc = ncoef(p)
    mono = [None] * nc
    mono[0] = SDA.const(p, syms, Poly.const(syms, 1))
    for i in range(1, nc):
        e = list(ex[i])
        v = 0 if e[0] else (1 if e[1] else 2)
        e[v] -= 1
        mono[i] = mono[index(*e)] * maps[v]
    out = [[Fraction(0)] * nc for _ in range(nc)]
    quarter = Fraction(-1, 4)
    for a in range(nc):
        for b in range(nc):
            poly = mono[a].c[b]
            if poly.is_zero():
                continue
            val = poly.subs_number("x0", quarter).subs_number("y0", quarter).subs_number("z0", quarter)
            out[b][a] = val.as_number() / (2 ** sum(ex[b]))
    return out


def octant_sign(e_out, e_in, octant):
    """Sign relating the (+,+,+) table to the table of another octant.  Reflecting axis v
    (s_v = -1) flips the sign of every coefficient with an odd exponent in v on both sides,
    so T_sigma[b][a] = sigma^(b+a) T[b][a]."""
    s = 1
    for v in range(3):
        if (octant >> v) & 1 and (e_out[v] + e_in[v]) % 2:
            s = -s
    return s


# ---- the harmonic basis -------------------------------------------------------------------
def free_coefficients(p):
    """Layout indices of the free coefficients of a harmonic expansion: those with z exponent
    c <= 1, (p + 1)^2 of them, in layout order.  The homogeneous parts of the multipole
    expansion (Eq. 2, the Legendre generating function) are harmonic polynomials, so every
    other coefficient follows from these by Laplace's equation."""
    return [i for i, e in enumerate(exponents(p)) if e[2] <= 1]


def harmonic_expansion(p):
    """X as sparse rows: X[i] = {free index j: Fraction} with a = X a[free] for every harmonic
    coefficient vector a.  Laplace's equation on the degree-n homogeneous part gives
    (c + 2)(c + 1) a[a, b, c + 2] = -(a + 2)(a + 1) a[a + 2, b, c] - (b + 2)(b + 1) a[a, b + 2, c],
    applied in order of increasing c.  Every step keeps the parity of each exponent, so X[i]
    only involves free coefficients of i's parity pattern."""
    ex = exponents(p)
    free = free_coefficients(p)
    X = [None] * len(ex)
    for j, i in enumerate(free):
        X[i] = {j: Fraction(1)}
    for i in sorted(range(len(ex)), key=lambda i: ex[i][2]):
        a, b, c = ex[i]
        if c <= 1:
            continue
        row = {}
        d = Fraction(c * (c - 1))
        for src, w in ((index(a + 2, b, c - 2), -Fraction((a + 2) * (a + 1)) / d),
                       (index(a, b + 2, c - 2), -Fraction((b + 2) * (b + 1)) / d)):
            for j, v in X[src].items():
                row[j] = row.get(j, Fraction(0)) + w * v
        X[i] = {j: v for j, v in row.items() if v != 0}
    return X


def m2m_harmonic_table(p, T=None):
    """The M2M table (m2m_scaled_table) for harmonic multipoles: rows restricted to the free
    coefficients and composed with the expansion X, so that the parent's free coefficients
    follow from the child's free coefficients alone (the M2M of a harmonic expansion is
    harmonic: it is the P2M of the same charges about another centre).  Dense nc x nc with
    zero rows and columns outside the free coefficients; column j of X becomes the layout
    column of free coefficient j, so the octant parity of an entry is that of its row and
    column layout exponents, as in the full table."""
    if T is None:
        T = m2m_scaled_table(p)
    nc = ncoef(p)
    free = free_coefficients(p)
    X = harmonic_expansion(p)
    out = [[Fraction(0)] * nc for _ in range(nc)]
    for b in free:
        acc = {}
        for a in range(nc):
            t = T[b][a]
            if t:
                for j, v in X[a].items():
                    acc[j] = acc.get(j, Fraction(0)) + t * v
        for j, v in acc.items():
            out[b][free[j]] = v
    return out
