"""Symbolic DA: truncated power series in three variables whose coefficients are
polynomials (exact rationals) in named symbols.

This is the build-time half of the method of Sec. 3: the same DA algorithms as
a numerical TPSA (product, binomial-series powers of an element that is not
infinitely small, composition) carried out on symbols instead of numbers, so
that every coefficient of an operator's result comes out as an explicit
expression.  Following the paper's variable substitution (Sec. 3, the r^2
trick), the constant part of an intermediate vector may be replaced by a new
symbol, which later steps inherit.

Pure Python (fractions.Fraction); no third-party algebra package.
"""
from fractions import Fraction


# ---- polynomials in symbols -----------------------------------------------------------
class Poly:
    """Sparse polynomial: dict exponent-tuple -> Fraction over a fixed symbol tuple."""

    __slots__ = ("syms", "t")

    def __init__(self, syms, terms=None):
        self.syms = syms
        self.t = terms if terms is not None else {}

    @staticmethod
    def const(syms, c):
        c = Fraction(c)
        return Poly(syms, {(0,) * len(syms): c} if c else {})

    @staticmethod
    def sym(syms, name, power=1, coef=1):
        e = [0] * len(syms)
        e[syms.index(name)] = power
        return Poly(syms, {tuple(e): Fraction(coef)})

    def is_zero(self):
        return not self.t

    def copy(self):
        return Poly(self.syms, dict(self.t))

    def __add__(self, o):
        r = dict(self.t)
        for e, c in o.t.items():
            v = r.get(e, 0) + c
            if v:
                r[e] = v
            else:
                r.pop(e, None)
        return Poly(self.syms, r)

    def iadd_scaled(self, o, s):
        """self += s * o (s a Fraction), in place."""
        r = self.t
        for e, c in o.t.items():
            v = r.get(e, 0) + s * c
            if v:
                r[e] = v
            else:
                r.pop(e, None)
        return self

    def scale(self, s):
        s = Fraction(s)
        if not s:
            return Poly(self.syms, {})
        return Poly(self.syms, {e: c * s for e, c in self.t.items()})

    def __mul__(self, o):
        if not self.t or not o.t:
            return Poly(self.syms, {})
        r = {}
        for e1, c1 in self.t.items():
            for e2, c2 in o.t.items():
                e = tuple(a + b for a, b in zip(e1, e2))
                v = r.get(e, 0) + c1 * c2
                if v:
                    r[e] = v
                else:
                    r.pop(e, None)
        return Poly(self.syms, r)

    def subs_number(self, name, value):
        """Substitute a rational number for one symbol."""
        k = self.syms.index(name)
        value = Fraction(value)
        r = {}
        for e, c in self.t.items():
            e2 = e[:k] + (0,) + e[k + 1:]
            v = r.get(e2, 0) + c * value ** e[k]
            if v:
                r[e2] = v
            else:
                r.pop(e2, None)
        return Poly(self.syms, r)

    def as_number(self):
        if not self.t:
            return Fraction(0)
        assert list(self.t) == [(0,) * len(self.syms)], "polynomial is not a constant"
        return self.t[(0,) * len(self.syms)]


# ---- DA layout (graded; x exponent descends, then y) -------------------------------------
def ncoef(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def index(a, b, c):
    n = a + b + c
    return n * (n + 1) * (n + 2) // 6 + (n - a) * (n - a + 1) // 2 + c


def exponents(p):
    out = [None] * ncoef(p)
    for n in range(p + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                c = n - a - b
                out[index(a, b, c)] = (a, b, c)
    return out


_MUL_CACHE = {}


def mul_table(p):
    """(i, j, k) for every pair of coefficients whose product stays within order p."""
    if p not in _MUL_CACHE:
        ex = exponents(p)
        tab = []
        for i, ei in enumerate(ex):
            for j, ej in enumerate(ex):
                if sum(ei) + sum(ej) <= p:
                    tab.append((i, j, index(ei[0] + ej[0], ei[1] + ej[1], ei[2] + ej[2])))
        _MUL_CACHE[p] = tab
    return _MUL_CACHE[p]


class SDA:
    """A DA vector of order p whose coefficients are Poly objects."""

    def __init__(self, p, syms, coef=None):
        self.p = p
        self.syms = syms
        self.c = coef if coef is not None else [Poly(syms) for _ in range(ncoef(p))]

    @staticmethod
    def const(p, syms, poly):
        v = SDA(p, syms)
        v.c[0] = poly
        return v

    @staticmethod
    def var(p, syms, v, const_poly=None):
        """const + d_v"""
        r = SDA(p, syms)
        if const_poly is not None:
            r.c[0] = const_poly
        if p >= 1:
            r.c[index(int(v == 0), int(v == 1), int(v == 2))] = Poly.const(syms, 1)
        return r

    def copy(self):
        return SDA(self.p, self.syms, [x.copy() for x in self.c])

    def __add__(self, o):
        return SDA(self.p, self.syms, [a + b for a, b in zip(self.c, o.c)])

    def scale_poly(self, s):
        return SDA(self.p, self.syms, [x * s for x in self.c])

    def __mul__(self, o):
        r = [Poly(self.syms) for _ in range(ncoef(self.p))]
        nz_a = [i for i, x in enumerate(self.c) if not x.is_zero()]
        nz_b = set(i for i, x in enumerate(o.c) if not x.is_zero())
        ex = exponents(self.p)
        for i in nz_a:
            ei = ex[i]
            oi = sum(ei)
            for j in nz_b:
                ej = ex[j]
                if oi + sum(ej) > self.p:
                    continue
                k = index(ei[0] + ej[0], ei[1] + ej[1], ei[2] + ej[2])
                prod = self.c[i] * o.c[j]
                r[k] = r[k] + prod
        return SDA(self.p, self.syms, r)

    def nilpotent_part(self):
        r = self.copy()
        r.c[0] = Poly(self.syms)
        return r

    def pow_unit(self, s):
        """(1 + t)^s for t = self (no constant part) by the binomial series, exact rationals."""
        assert self.c[0].is_zero()
        s = Fraction(s)
        acc = SDA.const(self.p, self.syms, Poly.const(self.syms, 1))
        term = SDA.const(self.p, self.syms, Poly.const(self.syms, 1))
        binom = Fraction(1)
        for k in range(1, self.p + 1):
            binom = binom * (s - (k - 1)) / k
            term = term * self
            acc = acc + term.scale_poly(Poly.const(self.syms, binom))
        return acc
