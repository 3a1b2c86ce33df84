"""Pins of the oracle's seven operators (Sec. 2, Eqs. 1-7) against facts fixed
by mathematics rather than by the oracle's own formulas:
  - P2M of a unit charge: the order-n part is |s|^n |d|^n P_n(cos gamma)
    (Legendre generating function), and the "-2 r.d" reading of Eq. 2;
  - every homogeneous part of a multipole or local expansion of 1/r is a
    harmonic polynomial (Kelvin transform of a harmonic function);
  - M2M maps the P2M about the child centre to the P2M about the parent centre
    exactly (the map M1 has no constant part);
  - L2L is the exact polynomial identity L'(x) = L(r0 + x), and leaves the
    top-order coefficients unchanged (Sec. 3.3);
  - M2L / P2L / M2P / L2P converge to the direct sum as the order grows;
  - low-order Taylor coefficients against SymPy series of the closed form.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle as O


def exps(p):
    return O.exponents(p).astype(np.int64)


def homog_part_eval(C, p, n, d):
    ex = exps(p)
    sel = ex.sum(1) == n
    return float(np.sum(C[sel] * np.prod(d[None, :] ** ex[sel], axis=1)))


def laplacian(C, p):
    """coefficients of the Laplacian of the polynomial C (order p -> p-2)."""
    ex = exps(p)
    ix = {tuple(e): i for i, e in enumerate(ex)}
    out = np.zeros(len(C))
    for i, e in enumerate(ex):
        for v in range(3):
            if e[v] >= 2:
                g = list(e)
                g[v] -= 2
                out[ix[tuple(g)]] += e[v] * (e[v] - 1) * C[i]
    return out


def assert_harmonic(C, p, rel=1e-12):
    lap = laplacian(C, p)
    ex = exps(p)
    for n in range(p - 1):
        sel_out = ex.sum(1) == n
        sel_in = ex.sum(1) == n + 2
        scale = np.abs(C[sel_in]).max() * (n + 2) ** 2 + 1e-300
        assert np.abs(lap[sel_out]).max() <= rel * scale, (n, np.abs(lap[sel_out]).max(), scale)


@pytest.mark.parametrize("p", [4, 8, 10])
def test_p2m_legendre_generating_function(p):
    rng = np.random.default_rng(10 + p)
    for _ in range(5):
        s = rng.uniform(-1, 1, 3)
        M = O.p2m(p, s[None, :], [1.0])
        d = rng.standard_normal(3)
        d *= 0.37 / np.linalg.norm(d)
        cosg = s @ d / (np.linalg.norm(s) * np.linalg.norm(d))
        for n in range(p + 1):
            ref = (np.linalg.norm(s) * np.linalg.norm(d)) ** n * eval_legendre(n, cosg)
            got = homog_part_eval(M, p, n, d)
            assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref)), (n, got, ref)


def test_p2m_sign_reading_reproduces_potential():
    """|d| phi_M(d) with d = r/r^2 must approach 1/|r - s| (the printed '+' sign would give 1/|r + s|)."""
    p = 10
    s = np.array([0.3, -0.2, 0.25])
    M = O.p2m(p, s[None, :], [1.0])
    r = np.array([2.0, 1.5, -1.0])
    phi, _ = O.m2p(p, M, r[None, :])
    assert abs(phi[0] - 1.0 / np.linalg.norm(r - s)) < 1e-8
    assert abs(phi[0] - 1.0 / np.linalg.norm(r + s)) > 1e-3


def test_p2m_against_symbolic_series():
    sp = pytest.importorskip("sympy")
    u, v, w, t = sp.symbols("u v w t")
    s = (sp.Rational(1, 3), sp.Rational(-1, 5), sp.Rational(2, 7))
    d = (t * u, t * v, t * w)
    expr = 1 / sp.sqrt(1 - 2 * sum(a * b for a, b in zip(s, d)) + sum(a * a for a in s) * sum(b * b for b in d))
    p = 4
    ser = sp.expand(sp.series(expr, t, 0, p + 1).removeO().subs(t, 1))
    poly = sp.Poly(ser, u, v, w)
    ref = {tuple(m): float(c) for m, c in poly.terms()}
    M = O.p2m(p, np.array([[float(x) for x in s]]), [1.0])
    for i, e in enumerate(exps(p)):
        assert abs(M[i] - ref.get(tuple(e), 0.0)) <= 1e-14 * (1 + abs(ref.get(tuple(e), 0.0)))


@pytest.mark.parametrize("p", [6, 10])
def test_harmonicity_of_all_expansions(p):
    rng = np.random.default_rng(20 + p)
    src = rng.uniform(-0.5, 0.5, (7, 3))
    q = rng.uniform(-1, 1, 7)
    M = O.p2m(p, src, q)
    assert_harmonic(M, p)
    Mp = O.m2m(p, M, np.array([0.5, -0.5, 0.5]))
    assert_harmonic(Mp, p)
    L = O.m2l(p, M, np.array([3.0, -2.0, 1.0]))
    assert_harmonic(L, p, rel=1e-11)
    L2 = O.p2l(p, np.array([3.0, -2.0, 1.0])[None, :] - src, q)
    assert_harmonic(L2, p, rel=1e-11)
    Lc = O.l2l(p, L, np.array([0.25, 0.25, -0.25]))
    assert_harmonic(Lc, p, rel=1e-11)


@pytest.mark.parametrize("p", [3, 8, 10])
def test_m2m_is_exact(p):
    rng = np.random.default_rng(30 + p)
    h = 1.0  # child box [-0.5,0.5]^3 around the child centre
    for oct_ in range(8):
        o = np.array([oct_ & 1, (oct_ >> 1) & 1, (oct_ >> 2) & 1])
        r0 = (0.5 - o) * h  # parent centre - child centre
        src = rng.uniform(-0.5, 0.5, (9, 3)) * h
        q = rng.uniform(-1, 1, 9)
        Mc = O.p2m(p, src, q)
        Mp = O.m2m(p, Mc, r0)
        ref = O.p2m(p, src - r0[None, :], q)
        assert np.abs(Mp - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("p", [4, 10])
def test_l2l_is_exact_polynomial_shift(p):
    rng = np.random.default_rng(40 + p)
    L = rng.standard_normal(O.ncoef(p))
    r0 = np.array([0.25, -0.25, 0.25])
    Lc = O.l2l(p, L, r0)
    for _ in range(5):
        x = rng.uniform(-0.25, 0.25, 3)
        assert abs(O.da_eval(p, Lc, x) - O.da_eval(p, L, x + r0)) <= 1e-12 * np.abs(L).sum()
    top = exps(p).sum(1) == p
    assert np.array_equal(Lc[top], L[top])  # Sec. 3.3: highest-order terms stay the same


def _direct_at(src, q, tgt):
    d = tgt[:, None, :] - src[None, :, :]
    r = np.linalg.norm(d, axis=2)
    phi = (q[None, :] / r).sum(1)
    E = (q[None, :, None] * d / r[:, :, None] ** 3).sum(1)
    return phi, E


def test_m2l_converges_to_direct_and_to_p2l():
    rng = np.random.default_rng(50)
    src = rng.uniform(-0.5, 0.5, (20, 3))
    q = rng.uniform(-1, 1, 20)
    r0 = np.array([2.0, 1.0, -2.0])  # well separated (one box in between)
    tgt = r0[None, :] + rng.uniform(-0.5, 0.5, (10, 3))
    phi_ref, E_ref = _direct_at(src, q, tgt)
    errs, errE, gap = [], [], []
    for p in [2, 4, 6, 8, 10]:
        M = O.p2m(p, src, q)
        L = O.m2l(p, M, r0)
        phi, E = O.l2p(p, L, tgt - r0[None, :])
        errs.append(np.abs(phi - phi_ref).max() / np.abs(phi_ref).max())
        errE.append(np.abs(E - E_ref).max() / np.abs(E_ref).max())
        Lp = O.p2l(p, r0[None, :] - src, q)
        phi2, _ = O.l2p(p, Lp, tgt - r0[None, :])
        gap.append(np.abs(phi - phi2).max() / np.abs(phi_ref).max())
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert all(b < a for a, b in zip(errE, errE[1:])), errE
    assert errs[-1] < 1e-5 and errE[-1] < 1e-4
    assert gap[-1] < gap[0] * 1e-2


def test_m2l_matrix_equals_composition():
    rng = np.random.default_rng(51)
    for p in [2, 6]:
        M = rng.standard_normal(O.ncoef(p))
        r0 = np.array([2.0, -3.0, 1.0])
        K = O.m2l_matrix(p, r0)
        assert np.allclose(K @ M, O.m2l(p, M, r0), rtol=1e-13, atol=1e-14 * np.abs(K @ M).max())


def test_m2l_against_symbolic_taylor():
    """Columns of the M2L map are the Taylor coefficients of (r0+u)^alpha/|r0+u|^(2|alpha|+1)."""
    sp = pytest.importorskip("sympy")
    u, v, w, t = sp.symbols("u v w t")
    r0 = (sp.Integer(2), sp.Integer(-1), sp.Integer(3))
    p = 3
    K = O.m2l_matrix(p, np.array([float(x) for x in r0]))
    ex = exps(p)
    X = [r0[0] + t * u, r0[1] + t * v, r0[2] + t * w]
    R2 = X[0] ** 2 + X[1] ** 2 + X[2] ** 2
    for a, e in enumerate(ex):
        f = X[0] ** int(e[0]) * X[1] ** int(e[1]) * X[2] ** int(e[2]) / R2 ** sp.Rational(2 * int(e.sum()) + 1, 2)
        ser = sp.expand(sp.series(f, t, 0, p + 1).removeO().subs(t, 1))
        poly = sp.Poly(ser, u, v, w)
        ref = {tuple(m): float(c) for m, c in poly.terms()}
        for b, eb in enumerate(ex):
            r = ref.get(tuple(eb), 0.0)
            assert abs(K[b, a] - r) <= 1e-14 * (1 + abs(r)), (a, b)


def test_m2p_converges_with_field():
    rng = np.random.default_rng(52)
    src = rng.uniform(-0.5, 0.5, (15, 3))
    q = rng.uniform(-1, 1, 15)
    tgt = np.array([[2.5, 0.3, -0.4], [-1.9, 2.2, 0.1], [0.2, 0.1, 3.0]])
    phi_ref, E_ref = _direct_at(src, q, tgt)
    prev = np.inf
    for p in [2, 4, 6, 8, 10]:
        M = O.p2m(p, src, q)
        phi, E = O.m2p(p, M, tgt)
        err = max(np.abs(phi - phi_ref).max() / np.abs(phi_ref).max(),
                  np.abs(E - E_ref).max() / np.abs(E_ref).max())
        assert err < prev
        prev = err
    assert prev < 1e-5


def test_l2p_field_is_minus_gradient():
    rng = np.random.default_rng(53)
    p = 7
    L = rng.standard_normal(O.ncoef(p))
    x = rng.uniform(-0.3, 0.3, (4, 3))
    phi, E = O.l2p(p, L, x)
    eps = 1e-6
    for k in range(3):
        dx = np.zeros(3)
        dx[k] = eps
        pp, _ = O.l2p(p, L, x + dx)
        pm, _ = O.l2p(p, L, x - dx)
        fd = -(pp - pm) / (2 * eps)
        assert np.allclose(E[:, k], fd, rtol=1e-6, atol=1e-6)
