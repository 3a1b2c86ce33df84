"""The numerical-DA form of the seven operators on the GPU (DAFMM_OP_NUMERICAL_DA): each
operator applied step by step with truncated power series arithmetic (Sec. 2, Appendix A),
one warp per instance -- the baseline the paper's generated code replaces (Sec. 3).  Both
forms compute the same truncated expansions, so in FP64 they must agree to rounding: per
order, the largest |difference| relative to the largest coefficient of that order within
1e-12 (the paper reports at most 3.69e-14 between its numerical DA and generated operators,
Table 2).  The numerical-DA results are also held to the oracle (the operators' definitions,
written independently on the CPU) and the M2L to the matrices of the K generation."""
import numpy as np
import pytest

import oracle as O
from paper_2508_02626_gb300 import binding as B

pytestmark = pytest.mark.gpu

DA = B.DAFMM_FP64 | B.DAFMM_OP_NUMERICAL_DA
TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.dafmm_create(0)
    yield c
    B.dafmm_destroy(c)


def per_order_rel(got, ref, p):
    n = O.exponents(p).sum(1)
    worst = 0.0
    for k in range(p + 1):
        s = n == k
        scale = np.abs(ref[..., s]).max()
        if scale > 0:
            worst = max(worst, np.abs(got[..., s] - ref[..., s]).max() / scale)
    return worst


@pytest.mark.parametrize("p", [0, 1, 2, 5, 8, 10])
def test_p2m_p2l_numerical_da(ctx, p):
    rng = np.random.default_rng(5000 + p)
    n, nc = 3000, O.ncoef(p)
    s = rng.uniform(-0.5, 0.5, (n, 3))
    q = rng.uniform(-1, 1, n)
    w = rng.uniform(-0.5, 0.5, (n, 3)) + np.array([2.0, -1.0, 3.0])
    for op, arg in ((B.dafmm_op_p2m, s), (B.dafmm_op_p2l, w)):
        gen, da = np.zeros((n, nc)), np.zeros((n, nc))
        op(ctx, p, B.DAFMM_FP64, arg, q, gen)
        op(ctx, p, DA, arg, q, da)
        assert per_order_rel(da, gen, p) <= TOL
    for i in range(0, n, 300):
        assert per_order_rel(da[i], O.p2l(p, w[i][None, :], [q[i]]), p) <= TOL


@pytest.mark.parametrize("p", [0, 2, 6, 10])
def test_l2p_m2p_numerical_da(ctx, p):
    rng = np.random.default_rng(6000 + p)
    n, nc = 2000, O.ncoef(p)
    C = rng.standard_normal((n, nc))
    x = rng.uniform(-0.5, 0.5, (n, 3))
    s = rng.uniform(-0.5, 0.5, (n, 3)) + np.array([-2.0, 3.0, 1.0])
    for op, arg in ((B.dafmm_op_l2p, x), (B.dafmm_op_m2p, s)):
        gen, da = np.zeros((n, 4)), np.zeros((n, 4))
        op(ctx, p, B.DAFMM_FP64, C, arg, gen)
        op(ctx, p, DA, C, arg, da)
        scale = np.abs(C).sum(1, keepdims=True) * (p + 1)
        assert (np.abs(da - gen) / scale).max() <= TOL
    for i in range(0, n, 400):  # M2P against the oracle: potential and E = -grad
        phi, E = O.m2p(p, C[i], s[i][None, :])
        sc = np.abs(C[i]).sum() * (p + 1)
        assert abs(da[i, 0] - phi[0]) <= TOL * sc
        assert np.abs(-da[i, 1:] - E[0]).max() <= TOL * sc


@pytest.mark.parametrize("p", [1, 4, 8, 10])
def test_m2m_l2l_numerical_da(ctx, p):
    rng = np.random.default_rng(7000 + p)
    n, nc = 256, O.ncoef(p)
    octs = rng.integers(0, 8, n).astype(np.int32)
    M = rng.standard_normal((n, nc))
    en = O.exponents(p).sum(1)
    for op in (B.dafmm_op_m2m, B.dafmm_op_l2l):
        gen, da = np.zeros((n, nc)), np.zeros((n, nc))
        op(ctx, p, B.DAFMM_FP64, octs, M, gen)
        op(ctx, p, DA, octs, M, da)
        assert per_order_rel(da, gen, p) <= TOL, op
    for i in range(0, n, 64):  # L2L against the oracle (Eq. 7, child width 1/2)
        o = np.array([octs[i] & 1, (octs[i] >> 1) & 1, (octs[i] >> 2) & 1])
        ref = O.l2l(p, M[i], (o - 0.5) * 0.5) / 2.0 ** en
        assert per_order_rel(da[i], ref, p) <= TOL


@pytest.mark.parametrize("p", [2, 6, 10])
def test_m2l_numerical_da(ctx, p):
    """Integer displacements against the GPU's M2L matrices (K generation), a non-integer one
    against the oracle's M2L (Eq. 5)."""
    rng = np.random.default_rng(8000 + p)
    nc = O.ncoef(p)
    vs = [[2, 0, 0], [3, -3, 3], [-2, 1, -3], [0, 2, -1]]
    M = rng.standard_normal((len(vs), nc))
    out = np.zeros((len(vs), nc))
    B.dafmm_op_m2l(ctx, p, DA, np.array(vs, dtype=np.float64), M, out)
    for i, v in enumerate(vs):
        K = np.zeros((nc, nc))
        B.dafmm_op_m2l_matrix(ctx, p, v, K)
        assert per_order_rel(out[i], K @ M[i], p) <= TOL, v
    r0 = np.array([[2.3, -1.7, 0.4]])
    out1 = np.zeros((1, nc))
    B.dafmm_op_m2l(ctx, p, DA, r0, M[:1], out1)
    assert per_order_rel(out1[0], O.m2l(p, M[0], r0[0]), p) <= TOL


def test_numerical_da_refusals(ctx):
    """Numerical DA is FP64 only, and dafmm_op_m2l has no generated form."""
    q = np.ones(4)
    s = np.zeros((4, 3))
    with pytest.raises(B.DafmmError) as e:
        B.dafmm_op_p2m(ctx, 4, B.DAFMM_FP32 | B.DAFMM_OP_NUMERICAL_DA, s, q, np.zeros((4, O.ncoef(4))))
    assert e.value.code == B.DAFMM_ERR_INVALID_ARG
    with pytest.raises(B.DafmmError) as e:
        B.dafmm_op_m2l(ctx, 4, B.DAFMM_FP64, np.full((4, 3), 2.0), np.zeros((4, O.ncoef(4))),
                       np.zeros((4, O.ncoef(4))))
    assert e.value.code == B.DAFMM_ERR_UNSUPPORTED
