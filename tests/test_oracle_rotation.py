"""Pins of the oracle's rotation-based M2L (Sec. 3.4).

The rotation Q of Sec. 3.4 (about x by atan2(z, y), then about z by atan2(sqrt(y^2+z^2), x))
must be orthogonal with determinant +1 and take r0 to (|r0|, 0, 0); composing a DA vector
with a linear map must agree with evaluating the polynomial at the mapped point; and the
rotated M2L must equal the plain Eq. 5 M2L for any displacement, since both compute the same
function (the Coulomb kernel is rotation invariant).  A rotation applied in the wrong sense
(Q instead of Q^T for the source expansion) must break that equality.
"""
import numpy as np
import pytest

import oracle as O

def _dirs():
    rng = np.random.default_rng(77)
    out = [np.array(v, float) for v in ((3.0, 0, 0), (-2.0, 0, 0), (0, 2.0, 0), (0, 0, -3.0), (2.0, -1.0, 0),
                                         (1.0, 0, 2.0), (-2.0, 3.0, -1.0), (3.0, 3.0, 3.0))]
    for _ in range(8):
        v = rng.normal(size=3)
        out.append(v / np.linalg.norm(v) * rng.uniform(2.0, 5.5))
    return out


def test_rotation_is_proper_and_aligns():
    for r0 in _dirs():
        Q = O.rotation(r0)
        assert np.allclose(Q @ Q.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(Q) - 1.0) < 1e-14
        assert np.allclose(Q @ r0, [np.linalg.norm(r0), 0.0, 0.0], atol=1e-13)


def test_linmap_matches_pointwise_evaluation():
    rng = np.random.default_rng(5)
    for p in (3, 7):
        a = rng.normal(size=O.ncoef(p))
        A = O.rotation(rng.normal(size=3))
        b = O.da_linmap(p, a, A)
        for _ in range(5):
            u = rng.uniform(-0.3, 0.3, 3)
            assert abs(O.da_eval(p, b, u) - O.da_eval(p, a, A @ u)) < 1e-13 * max(1.0, np.abs(a).sum())
        # round trip through Q and Q^T returns the vector (degree by degree, exactly up to rounding)
        back = O.da_linmap(p, b, A.T)
        assert np.allclose(back, a, rtol=0, atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10])
def test_rotated_m2l_equals_eq5(p):
    rng = np.random.default_rng(100 + p)
    nc = O.ncoef(p)
    for r0 in _dirs():
        M = rng.normal(size=nc) / (1.0 + O.exponents(p).sum(axis=1))
        ref = O.m2l(p, M, r0)
        got = O.m2l_rot(p, M, r0)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (p, r0)


def test_wrong_rotation_sense_is_detected():
    p = 6
    rng = np.random.default_rng(3)
    M = rng.normal(size=O.ncoef(p))
    r0 = np.array([-2.0, 3.0, -1.0])
    Q = O.rotation(r0)
    ax = np.array([np.linalg.norm(r0), 0.0, 0.0])
    # the planted mistake: Q (instead of Q^T) for the source expansion
    wrong = O.da_linmap(p, O.m2l(p, O.da_linmap(p, M, Q), ax), Q)
    right = O.da_linmap(p, O.m2l(p, O.da_linmap(p, M, Q.T), ax), Q)
    ref = O.m2l(p, M, r0)
    assert np.abs(right - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()


def test_fmm_with_rotated_m2l_equals_matrix_m2l():
    rng = np.random.default_rng(9)
    n = 1500
    x = rng.random((n, 3))
    q = rng.uniform(-1, 1, n)
    dom = (0.0, 0.0, 0.0, 1.0)
    a_phi, a_E = O.fmm(x, q, dom, 5, uniform_depth=3, m2l_mode=1)
    b_phi, b_E = O.fmm(x, q, dom, 5, uniform_depth=3, m2l_mode=2)
    assert np.abs(b_phi - a_phi).max() <= 1e-12 * np.abs(a_phi).max()
    assert np.abs(b_E - a_E).max() <= 1e-11 * np.abs(a_E).max()
