"""Pins of the oracle's numerical DA (Appendix A) against values fixed by the
paper and by mathematics: Table 1, closed-form Taylor series, and symbolic
differentiation / expansion done independently by SymPy."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def idx_of(order):
    ex = O.exponents(order)
    return {tuple(int(v) for v in e): i for i, e in enumerate(ex)}


def test_layout_graded_and_ordered():
    # D1 layout: graded by order; inside an order x exponent descends, then y (Table 1 order)
    ex = O.exponents(3)
    assert O.ncoef(3) == 20 and len(ex) == 20
    expect = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0),
              (0, 1, 1), (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2),
              (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]
    assert [tuple(e) for e in ex] == expect
    for p in range(11):
        assert O.ncoef(p) == (p + 1) * (p + 2) * (p + 3) // 6


def test_table1_rinv_at_111():
    """Table 1: the DA column for 1/r at (1,1,1), order 2."""
    v = O.da_rinv(2, [1.0, 1.0, 1.0])
    ix = idx_of(2)
    for a, b, c, val in read_golden("table1_rinv_at_111_order2.txt"):
        got = v[ix[(int(a), int(b), int(c))]]
        assert abs(got - val) <= 1e-16 + 2e-16 * abs(val), (a, b, c, got, val)


@pytest.mark.parametrize("a", [0.7, 1.0, 2.5])
def test_rinv_on_axis_closed_form(a):
    """1/|(a,0,0)+d|: the d_x^n coefficient is (-1)^n / a^(n+1); the d_y^2
    coefficient is -1/(2 a^3); the d_x d_y^2 coefficient is 3/(2 a^4)."""
    p = 10
    v = O.da_rinv(p, [a, 0.0, 0.0])
    ix = idx_of(p)
    for n in range(p + 1):
        ref = (-1) ** n / a ** (n + 1)
        assert abs(v[ix[(n, 0, 0)]] - ref) <= 1e-12 * abs(ref)
    assert abs(v[ix[(0, 2, 0)]] + 0.5 / a ** 3) <= 1e-12 / a ** 3
    assert abs(v[ix[(1, 2, 0)]] - 1.5 / a ** 4) <= 1e-12 / a ** 4
    # odd powers of d_y or d_z vanish by symmetry
    for (i, j, k), t in ix.items():
        if j % 2 or k % 2:
            assert v[t] == 0.0 or abs(v[t]) < 1e-15


def test_rinv_against_symbolic_derivatives():
    """Taylor coefficient of 1/|x0+d| at d^alpha = (d/dx)^alpha (1/r) / alpha!  (SymPy, exact)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    f = 1 / sp.sqrt(x ** 2 + y ** 2 + z ** 2)
    pt = (sp.Rational(3, 10), sp.Rational(-7, 10), sp.Rational(11, 10))
    p = 5
    v = O.da_rinv(p, [float(c) for c in pt])
    for i, (a, b, c) in enumerate(O.exponents(p)):
        d = sp.diff(f, x, int(a), y, int(b), z, int(c)) if (a + b + c) else f
        ref = float(d.subs({x: pt[0], y: pt[1], z: pt[2]}) / (math.factorial(a) * math.factorial(b) * math.factorial(c)))
        assert abs(v[i] - ref) <= 1e-14 * max(1.0, abs(ref)), (a, b, c, v[i], ref)


def _rand_da(rng, p, const=None):
    a = rng.standard_normal(O.ncoef(p))
    if const is not None:
        a[0] = const
    return a


def _to_sympy(a, p, syms):
    ex = O.exponents(p)
    return sum(float(a[i]) * syms[0] ** int(e[0]) * syms[1] ** int(e[1]) * syms[2] ** int(e[2])
               for i, e in enumerate(ex))


def _truncate(expr, p, syms):
    import sympy as sp
    poly = sp.Poly(sp.expand(expr), *syms)
    out = {}
    for mon, coef in poly.terms():
        if sum(mon) <= p:
            out[tuple(mon)] = float(coef)
    return out


def test_mul_and_compose_against_symbolic_expansion():
    sp = pytest.importorskip("sympy")
    syms = sp.symbols("u v w")
    rng = np.random.default_rng(5)
    p = 4
    ix = idx_of(p)
    a, b = _rand_da(rng, p), _rand_da(rng, p)
    prod = O.da_mul(p, a, b)
    ref = _truncate(_to_sympy(a, p, syms) * _to_sympy(b, p, syms), p, syms)
    for mon, i in ix.items():
        assert abs(prod[i] - ref.get(mon, 0.0)) <= 1e-12 * (1 + abs(ref.get(mon, 0.0)))
    # composition with a map that has a constant part (the M2L case)
    f = _rand_da(rng, 3)
    g = np.concatenate([_rand_da(rng, p) * 0.5 for _ in range(3)])
    comp = O.da_compose(3, f, p, g)
    gs = [_to_sympy(g[k * O.ncoef(p):(k + 1) * O.ncoef(p)], p, syms) for k in range(3)]
    fe = _to_sympy(f, 3, sp.symbols("X Y Z"))
    X, Y, Z = sp.symbols("X Y Z")
    ref = _truncate(fe.subs({X: gs[0], Y: gs[1], Z: gs[2]}, simultaneous=True), p, syms)
    for mon, i in ix.items():
        assert abs(comp[i] - ref.get(mon, 0.0)) <= 1e-11 * (1 + abs(ref.get(mon, 0.0))), mon


def test_deriv_against_symbolic():
    sp = pytest.importorskip("sympy")
    syms = sp.symbols("u v w")
    rng = np.random.default_rng(6)
    p = 5
    a = _rand_da(rng, p)
    ae = _to_sympy(a, p, syms)
    ix = idx_of(p)
    for v in range(3):
        d = O.da_deriv(p, a, v)
        ref = _truncate(sp.diff(ae, syms[v]), p, syms)
        for mon, i in ix.items():
            assert abs(d[i] - ref.get(mon, 0.0)) <= 1e-12 * (1 + abs(ref.get(mon, 0.0)))


@pytest.mark.parametrize("s", [-1.0, -0.5, 0.5, -1.5])
def test_pow_series_against_symbolic(s):
    """a^s by the binomial series equals the Taylor expansion of the power of the polynomial."""
    sp = pytest.importorskip("sympy")
    syms = sp.symbols("u v w")
    rng = np.random.default_rng(7)
    p = 4
    a = _rand_da(rng, p, const=1.7)
    a[1:] *= 0.3
    got = O.da_pow(p, a, s)
    t = sp.symbols("t")
    ae = _to_sympy(a, p, [t * q for q in syms])
    ser = sp.series(ae ** sp.Rational(s).limit_denominator(4), t, 0, p + 1).removeO().subs(t, 1)
    ref = _truncate(ser, p, syms)
    ix = idx_of(p)
    for mon, i in ix.items():
        assert abs(got[i] - ref.get(mon, 0.0)) <= 1e-12 * (1 + abs(ref.get(mon, 0.0))), mon


def test_eval_matches_polynomial():
    rng = np.random.default_rng(8)
    p = 6
    a = _rand_da(rng, p)
    x = rng.standard_normal(3)
    ex = O.exponents(p)
    ref = sum(a[i] * x[0] ** e[0] * x[1] ** e[1] * x[2] ** e[2] for i, e in enumerate(ex))
    assert abs(O.da_eval(p, a, x) - ref) <= 1e-12 * (1 + abs(ref))
