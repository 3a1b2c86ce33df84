"""The harmonic basis of the FP32 mode's M2L, pinned with the oracle (no code shared with the
kernels).

Facts pinned:
  * the homogeneous parts of a P2M multipole expansion (Eq. 2) are harmonic polynomials in d:
    the coefficients with z exponent c >= 2 follow from those with c <= 1 by Laplace's equation
    (c + 2)(c + 1) a[a, b, c + 2] = -(a + 2)(a + 1) a[a + 2, b, c] - (b + 2)(b + 1) a[a, b + 2, c];
  * so are those of the local expansions the M2L (Eq. 5) produces;
  * hence the M2L restricted to the (p + 1)^2 free coefficients -- K^_v's free rows composed
    with the expansion X from the free coefficients -- followed by X reproduces K^_v M;
  * the free coefficients are (p + 1)^2 in number and, in the coefficient layout, are (n, 0, 0),
    (n - 1, 1, 0), (n - 1, 0, 1), (n - 2, 2, 0), ... within degree n.
A planted mistake (a non-harmonic vector) fails the harmonic check, so the check has teeth."""
import numpy as np
import pytest

import oracle as O


def basis(p):
    E = O.exponents(p)
    idx = {tuple(int(v) for v in e): i for i, e in enumerate(E)}
    free = [i for i, e in enumerate(E) if e[2] <= 1]
    X = np.zeros((len(E), len(free)))
    for j, i in enumerate(free):
        X[i, j] = 1.0
    for i in sorted(range(len(E)), key=lambda i: E[i][2]):
        a, b, c = (int(v) for v in E[i])
        if c <= 1:
            continue
        X[i] = -((a + 2) * (a + 1) * X[idx[(a + 2, b, c - 2)]] + (b + 2) * (b + 1) * X[idx[(a, b + 2, c - 2)]]) / (
            c * (c - 1))
    return E, free, X


def harmonic_residual(v, free, X):
    return np.abs(X @ v[free] - v).max() / np.abs(v).max()


def free_index(k):
    """The layout index of free coefficient k (the kernels' harm_full_index, restated)."""
    n = int(np.floor(np.sqrt(k)))
    while (n + 1) ** 2 <= k:
        n += 1
    r = k - n * n
    a = n - (r + 1) // 2
    c = 1 if r > 0 and r % 2 == 0 else 0
    b = n - a - c
    return n * (n + 1) * (n + 2) // 6 + (b + c) * (b + c + 1) // 2 + c


@pytest.mark.parametrize("p", range(0, 11))
def test_free_coefficients(p):
    E, free, _ = basis(p)
    assert len(free) == (p + 1) ** 2
    assert free == [free_index(k) for k in range((p + 1) ** 2)]


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10])
def test_multipoles_and_locals_are_harmonic(p):
    E, free, X = basis(p)
    rng = np.random.default_rng(40 + p)
    M = O.p2m(p, rng.uniform(-0.5, 0.5, (40, 3)), rng.uniform(-1, 1, 40))
    assert harmonic_residual(M, free, X) < 1e-13
    for v in ([2, 0, 0], [3, -3, 3], [-2, 1, -3], [0, 2, -1]):
        L = O.m2l_matrix(p, np.array(v, float)) @ M
        assert harmonic_residual(L, free, X) < 1e-13
    # planted mistake: a generic coefficient vector is not harmonic
    assert harmonic_residual(rng.standard_normal(len(E)), free, X) > 1e-2


@pytest.mark.parametrize("p", [2, 5, 8, 10])
def test_reduced_m2l_reproduces_the_dense_one(p):
    E, free, X = basis(p)
    rng = np.random.default_rng(70 + p)
    M = O.p2m(p, rng.uniform(-0.5, 0.5, (40, 3)), rng.uniform(-1, 1, 40))
    for v in ([2, 0, 0], [3, -3, 3], [-2, 1, -3]):
        K = O.m2l_matrix(p, np.array(v, float))
        L = K @ M
        Kh = K[free] @ X
        assert Kh.shape == ((p + 1) ** 2, (p + 1) ** 2)
        Lh = X @ (Kh @ M[free])
        assert np.abs(Lh - L).max() <= 1e-13 * np.abs(L).max()
