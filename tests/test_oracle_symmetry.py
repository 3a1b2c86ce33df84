"""The octahedral symmetry of the M2L matrices (the 48 signed axis permutations map the 316
displacements onto 16 classes), checked on the oracle's matrices.

For a signed permutation g, (g w)_d = sigma_d w_{pi(d)}, the kernel 1/|w| is invariant, and
a monomial transforms as (g u)^a = s(a) u^{gamma(a)} with s(a) = prod_d sigma_d^{a_d} and
gamma(a)_{pi(d)} = a_d.  Hence K_{g c}[b][a] = s(a) s(b) K_c[gamma(b)][gamma(a)]: every
matrix follows from the one of its class representative c = (|v| sorted descending).  The
GPU generates the 16 representatives and expands the rest with this rule."""
import itertools

import numpy as np
import pytest

import oracle as O


def symmetry_of(v):
    """(c, pi, sigma) with v_d = sigma_d c_{pi(d)}, c = |v| sorted descending."""
    av = np.abs(np.asarray(v))
    order = sorted(range(3), key=lambda d: (-av[d], d))  # c_j = |v_{order[j]}|
    c = tuple(int(av[d]) for d in order)
    pi = [0, 0, 0]
    for j, d in enumerate(order):
        pi[d] = j
    sigma = [1 if v[d] >= 0 else -1 for d in range(3)]
    return c, pi, sigma


def expand(Kc, p, pi, sigma):
    ex = O.exponents(p)
    index = {tuple(e): i for i, e in enumerate(ex)}
    nc = len(ex)
    g = np.zeros(nc, dtype=int)
    sgn = np.zeros(nc)
    for i, e in enumerate(ex):
        ge = [0, 0, 0]
        for d in range(3):
            ge[pi[d]] = e[d]
        g[i] = index[tuple(ge)]
        sgn[i] = np.prod([sigma[d] ** e[d] for d in range(3)])
    return sgn[:, None] * sgn[None, :] * Kc[np.ix_(g, g)]


def test_sixteen_classes():
    vs = [v for v in itertools.product(range(-3, 4), repeat=3) if max(map(abs, v)) > 1]
    assert len(vs) == 316
    assert len({symmetry_of(v)[0] for v in vs}) == 16


@pytest.mark.parametrize("p", [3, 6, 8])
def test_expansion_reproduces_every_matrix(p):
    rng = np.random.default_rng(p)
    vs = [v for v in itertools.product(range(-3, 4), repeat=3) if max(map(abs, v)) > 1]
    cache = {}
    for k in rng.choice(len(vs), 40, replace=False):
        v = vs[k]
        c, pi, sigma = symmetry_of(v)
        if c not in cache:
            cache[c] = O.m2l_matrix(p, np.array(c, float))
        Kv = O.m2l_matrix(p, np.array(v, float))
        Ke = expand(cache[c], p, pi, sigma)
        assert np.abs(Ke - Kv).max() <= 1e-12 * np.abs(Kv).max(), v
    # a wrong sign or the inverse of a 3-cycle permutation does not reproduce the matrices
    v = (1, -3, 2)
    c, pi, sigma = symmetry_of(v)
    Kv = O.m2l_matrix(p, np.array(v, float))
    Kc = O.m2l_matrix(p, np.array(c, float))
    assert np.abs(expand(Kc, p, pi, [1, 1, 1]) - Kv).max() > 1e-3 * np.abs(Kv).max()
    inv = [pi.index(j) for j in range(3)]
    assert np.abs(expand(Kc, p, inv, sigma) - Kv).max() > 1e-3 * np.abs(Kv).max()
