"""The generated straight-line operators (host build) against the oracle, following the
paper's verification protocol (Sec. 3): many random instances, compared order by order;
per order the largest absolute difference |delta| and the relative difference of that
coefficient are recorded.  The paper observed |delta_r| <= 3.69e-14 between its generated
and numerical-DA operators (Table 2); the bound used here is 1e-12 relative to the largest
coefficient of the order (FP64) and 2e-5 (FP32)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2508_02626_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hc():
    gen_dir = _build.generate()
    d = tempfile.mkdtemp(prefix="dafmm_hc_")
    so = os.path.join(d, "hc.so")
    src = os.path.join(ROOT, "tests", "gen_host_check.cpp")
    inc = os.path.dirname(gen_dir)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                           "-I", inc, "-o", so, src])
    lib = ctypes.CDLL(so)
    D = ctypes.POINTER(ctypes.c_double)
    for nm, args in {"hc_p2m": [ctypes.c_int, ctypes.c_int, D, ctypes.c_double, D, ctypes.c_int],
                     "hc_p2mh": [ctypes.c_int, ctypes.c_int, D, ctypes.c_double, D, ctypes.c_int],
                     "hc_p2l": [ctypes.c_int, ctypes.c_int, D, ctypes.c_double, D, ctypes.c_int],
                     "hc_l2p": [ctypes.c_int, ctypes.c_int, D, D, D, ctypes.c_int],
                     "hc_m2p": [ctypes.c_int, ctypes.c_int, D, D, D, ctypes.c_int],
                     "hc_m2lmap": [ctypes.c_int, D, D, D],
                     "hc_shift": [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, ctypes.c_int]}.items():
        getattr(lib, nm).argtypes = args
        getattr(lib, nm).restype = ctypes.c_int
    return lib


def P(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def per_order_rel(got, ref, p):
    ex = O.exponents(p)
    n = ex.sum(1)
    worst = 0.0
    for k in range(p + 1):
        s = n == k
        scale = np.abs(ref[..., s]).max()
        if scale == 0:
            continue
        worst = max(worst, np.abs(got[..., s] - ref[..., s]).max() / scale)
    return worst


ORDERS = [0, 1, 2, 3, 5, 6, 8, 10]


@pytest.mark.parametrize("p", ORDERS)
def test_generated_p2m_p2l(hc, p):
    rng = np.random.default_rng(100 + p)
    nc = O.ncoef(p)
    n = 300
    for prec, tol in ((64, 1e-12), (32, 2e-5)):
        g_m, r_m, g_l, r_l = [], [], [], []
        for _ in range(n):
            s = rng.uniform(-0.5, 0.5, 3)  # charge inside the unit box (Sec. 3 setup)
            q = rng.uniform(-1, 1)
            out = np.zeros(nc)
            assert hc.hc_p2m(p, prec, P(s), q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
            g_m.append(out)
            r_m.append(O.p2m(p, s[None, :], [q]))
            w = rng.uniform(-0.5, 0.5, 3) + np.array([2.0, -1.0, 2.0])  # source two boxes away
            out2 = np.zeros(nc)
            assert hc.hc_p2l(p, prec, P(w), q, out2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
            g_l.append(out2)
            r_l.append(O.p2l(p, w[None, :], [q]))
        assert per_order_rel(np.array(g_m), np.array(r_m), p) <= tol
        assert per_order_rel(np.array(g_l), np.array(r_l), p) <= tol


@pytest.mark.parametrize("p", ORDERS)
def test_generated_l2p_m2p(hc, p):
    rng = np.random.default_rng(200 + p)
    nc = O.ncoef(p)
    for prec, tol in ((64, 1e-12), (32, 2e-5)):
        for _ in range(40):
            C = rng.standard_normal(nc)
            x = rng.uniform(-0.5, 0.5, 3)
            res = np.zeros(4)
            assert hc.hc_l2p(p, prec, P(C), P(x), res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
            phi, E = O.l2p(p, C, x[None, :])
            sc = np.abs(C).sum()
            assert abs(res[0] - phi[0]) <= tol * sc
            assert np.abs(-res[1:] - E[0]).max() <= tol * sc * (p + 1)
            s = rng.uniform(-0.5, 0.5, 3) + np.array([-2.0, 2.0, 1.0])
            res = np.zeros(4)
            assert hc.hc_m2p(p, prec, P(C), P(s), res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
            phi, E = O.m2p(p, C, s[None, :])
            assert abs(res[0] - phi[0]) <= tol * sc
            assert np.abs(-res[1:] - E[0]).max() <= tol * sc * (p + 1)


@pytest.mark.parametrize("p", ORDERS)
def test_generated_m2l_map(hc, p):
    nc = O.ncoef(p)
    for v in ([2.0, 0.0, -3.0], [3.0, 3.0, 3.0], [-2.0, 1.0, 0.0]):
        v = np.array(v)
        inv, isq = np.zeros(nc), np.zeros(nc)
        assert hc.hc_m2lmap(p, P(v), inv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            isq.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
        rho = 1.0 / (v @ v)
        sR, mp = O.m2l_map(p, v)
        assert np.allclose(np.sqrt(rho) * isq, sR, rtol=1e-13, atol=1e-15 * np.abs(sR).max())
        # M2_k = (v_k + u_k) R with R = rho * inv
        R = rho * inv
        ex = O.exponents(p)
        ix = {tuple(e): i for i, e in enumerate(ex)}
        for k in range(3):
            m2 = v[k] * R
            for i, e in enumerate(ex):
                if e.sum() < p:
                    f = list(e)
                    f[k] += 1
                    m2[ix[tuple(f)]] += R[i]
            assert np.allclose(m2, mp[k], rtol=1e-13, atol=1e-15 * np.abs(mp[k]).max())


@pytest.mark.parametrize("p", ORDERS)
def test_generated_shift_tables(hc, p):
    """M2M and L2L tables (scaled variables, octant signs) against the oracle's operators."""
    rng = np.random.default_rng(300 + p)
    nc = O.ncoef(p)
    ex = O.exponents(p)
    n = ex.sum(1)
    for c in range(8):
        o = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        M = rng.standard_normal(nc)
        out = np.zeros(nc)
        assert hc.hc_shift(p, 0, c, P(M), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
        # child width 1, parent width 2: M~' = M' / 2^|b|
        ref = O.m2m(p, M, 0.5 - o) / 2.0 ** n
        assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()
        L = rng.standard_normal(nc)
        out = np.zeros(nc)
        assert hc.hc_shift(p, 1, c, P(L), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
        # parent width 1, child width 1/2: L~' = L' * (1/2)^|b|
        ref = O.l2l(p, L, (o - 0.5) * 0.5) / 2.0 ** n
        assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


def free_layout(p):
    """Layout indices of the coefficients of z exponent <= 1, from the oracle's exponents."""
    return [i for i, e in enumerate(O.exponents(p)) if e[2] <= 1]


@pytest.mark.parametrize("p", ORDERS)
def test_generated_harmonic_p2m(hc, p):
    """The harmonic-basis P2M emits exactly the oracle P2M's coefficients of z exponent <= 1,
    (p + 1)^2 of them, in layout order."""
    rng = np.random.default_rng(400 + p)
    free = free_layout(p)
    nh = (p + 1) ** 2
    assert len(free) == nh
    for prec, tol in ((64, 1e-12), (32, 2e-5)):
        got, ref = [], []
        for _ in range(200):
            s = rng.uniform(-0.5, 0.5, 3)
            q = rng.uniform(-1, 1)
            out = np.zeros(nh)
            assert hc.hc_p2mh(p, prec, P(s), q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nh) == 0
            full = np.zeros(O.ncoef(p))
            full[free] = out
            got.append(full)
            r = np.array(O.p2m(p, s[None, :], [q]))
            r[[i for i in range(O.ncoef(p)) if i not in set(free)]] = 0.0
            ref.append(r)
        assert per_order_rel(np.array(got), np.array(ref), p) <= tol


@pytest.mark.parametrize("p", ORDERS)
def test_generated_harmonic_m2m_table(hc, p):
    """The M2M table of harmonic multipoles: from the child's free coefficients alone it gives
    the parent's free coefficients of the oracle's M2M (scaled variables, every octant), and it
    reads and writes nothing else.  A generic (non-harmonic) child vector gives a different
    result from the full table, so the composition with Laplace's equation is what makes it
    right."""
    rng = np.random.default_rng(500 + p)
    nc = O.ncoef(p)
    ex = O.exponents(p)
    n = ex.sum(1)
    free = free_layout(p)
    other = [i for i in range(nc) if i not in set(free)]
    for c in range(8):
        o = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        M = O.p2m(p, rng.uniform(-0.5, 0.5, (30, 3)), rng.uniform(-1, 1, 30))
        Mf = np.array(M, dtype=float)
        Mf[other] = np.nan  # reading a non-free coefficient would show up as NaN
        out = np.zeros(nc)
        assert hc.hc_shift(p, 2, c, P(Mf),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
        ref = O.m2m(p, M, 0.5 - o) / 2.0 ** n
        assert np.all(np.isfinite(out))
        assert np.abs(out[free] - ref[free]).max() <= 1e-13 * np.abs(ref).max()
        assert np.all(out[other] == 0.0)
    if p >= 3:  # (up to p = 2 no free row of the full table reads a coefficient with c >= 2)
        G = rng.standard_normal(nc)
        full, harm = np.zeros(nc), np.zeros(nc)
        assert hc.hc_shift(p, 0, 0, P(G), full.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
        assert hc.hc_shift(p, 2, 0, P(G), harm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nc) == 0
        assert np.abs(full[free] - harm[free]).max() > 1e-3 * np.abs(full).max()
