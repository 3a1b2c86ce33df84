"""The FP64 M2L by rotation (Sec. 3.4) on the GPU, through the C ABI.

With DAFMM_OPT_M2L_ROTATION = 1 (the default from p = 4) the FP64 evaluation of a uniform tree rotates each source
expansion so that the displacement lies on the x axis, applies Eq. 5 along the axis and
rotates back.  The operator is the same linear map as the dense K^_v matrix, so the result
must equal the oracle FMM on the same tree up to rounding (relative L2 1e-12, the FP64 bound
of the other parity tests), and the oracle's own rotation-based traversal (mode 2) as well.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_02626_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.Context(0)
    B.dafmm_set_option(c.h, B.DAFMM_OPT_M2L_ROTATION, 1)
    yield c
    c.close()


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def run(ctx, x, q, dom, depth, p):
    n = len(q)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    tree = ctx.build_tree(xt, qt, domain=dom, uniform_depth=depth)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree.eval(p, phi, E, precision="fp64")
    B.dafmm_sync(ctx.h)
    tree.free()
    return phi.cpu().numpy(), E.cpu().numpy()


@pytest.mark.parametrize("p,depth", [(2, 3), (4, 3), (6, 3), (8, 3), (10, 2), (10, 3)])
def test_rotated_m2l_matches_oracle(ctx, p, depth):
    rng = np.random.default_rng(40 + p + depth)
    n = 6000
    x = rng.random((n, 3))
    q = rng.uniform(-1, 1, n)
    dom = (0.0, 0.0, 0.0, 1.0)
    phi, E = run(ctx, x, q, dom, depth, p)
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=depth)
    assert rel(phi, ref_phi) <= 1e-12, rel(phi, ref_phi)
    assert rel(E, ref_E) <= 1e-11, rel(E, ref_E)


def test_rotated_m2l_matches_oracle_rotation_and_dense_gpu(ctx):
    rng = np.random.default_rng(7)
    n = 3000
    x = rng.random((n, 3)) * 2.0 - 1.0
    q = rng.uniform(-1, 1, n)
    dom = (-1.0, -1.0, -1.0, 2.0)
    p, depth = 6, 3
    phi, E = run(ctx, x, q, dom, depth, p)
    rot_phi, rot_E = O.fmm(x, q, dom, p, uniform_depth=depth, m2l_mode=2)
    assert rel(phi, rot_phi) <= 1e-12
    assert rel(E, rot_E) <= 1e-11
    plain = B.Context(0)
    B.dafmm_set_option(plain.h, B.DAFMM_OPT_M2L_ROTATION, 0)
    try:
        d_phi, d_E = run(plain, x, q, dom, depth, p)
    finally:
        plain.close()
    assert rel(phi, d_phi) <= 1e-13
    assert rel(E, d_E) <= 1e-12


def test_rotation_option_values(ctx):
    with pytest.raises(Exception):
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_ROTATION, 2)


def test_rotated_m2l_adaptive_forest(ctx):
    """Adaptive trees: the V-list pairs of a level have the same integer box displacements, so
    the rotation tables serve them too; a two-member forest of clustered points."""
    rng = np.random.default_rng(11)
    parts = []
    for m in range(2):
        c = rng.random((4, 3))
        x = c[rng.integers(0, 4, 5000)] + 0.05 * rng.normal(size=(5000, 3))
        parts.append(x)
    q = [rng.uniform(-1, 1, len(x)) for x in parts]
    xyz = np.concatenate(parts)
    qq = np.concatenate(q)
    offs = np.array([0, len(parts[0]), len(xyz)], dtype=np.int64)
    p = 6

    def run_forest(c):
        tree = c.build_forest(torch.from_numpy(xyz).cuda(), torch.from_numpy(qq).cuda(), offs, max_leaf=32)
        phi = torch.empty(len(qq), dtype=torch.float64, device="cuda")
        E = torch.empty((len(qq), 3), dtype=torch.float64, device="cuda")
        tree.eval(p, phi, E, precision="fp64")
        B.dafmm_sync(c.h)
        _, doms = tree.forest()
        tree.free()
        return phi.cpu().numpy(), E.cpu().numpy(), doms

    phi, E, doms = run_forest(ctx)
    plain = B.Context(0)
    B.dafmm_set_option(plain.h, B.DAFMM_OPT_M2L_ROTATION, 0)
    try:
        d_phi, d_E, _ = run_forest(plain)
    finally:
        plain.close()
    assert rel(phi, d_phi) <= 1e-13
    assert rel(E, d_E) <= 1e-12
    # each member against the oracle's adaptive FMM on the member's own root cube
    for m in range(2):
        a, b = offs[m], offs[m + 1]
        ref_phi, ref_E = O.fmm(xyz[a:b], qq[a:b], doms[m], p, max_leaf=32)
        assert rel(phi[a:b], ref_phi) <= 1e-12, (m, rel(phi[a:b], ref_phi))
        assert rel(E[a:b], ref_E) <= 1e-11


@pytest.mark.parametrize("p", [3, 4, 8, 10])
def test_harmonic_rotation_matches_full_lists(ctx, p):
    """The rotation in its harmonic form (the default: only the outputs of z exponent <= 1 of
    each step, the others restored by Laplace's equation before the last x-step and once per
    target) against the full task lists, FP64 and float-float: the same result up to rounding."""
    rng = np.random.default_rng(90 + p)
    n = 6000
    x = rng.random((n, 3))
    q = rng.uniform(-1, 1, n)
    dom = (0.0, 0.0, 0.0, 1.0)
    for prec, tol in (("fp64", 1e-13), ("ff", 1e-12)):
        out = {}
        for harm in (1, 0):
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, harm)
            try:
                xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
                tree = ctx.build_tree(xt, qt, domain=dom, uniform_depth=3)
                phi = torch.empty(n, dtype=torch.float64, device="cuda")
                E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
                tree.eval(p, phi, E, precision=prec)
                B.dafmm_sync(ctx.h)
                tree.free()
                out[harm] = (phi.cpu().numpy(), E.cpu().numpy())
            finally:
                B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, 1)
        assert rel(out[1][0], out[0][0]) <= tol, (prec, rel(out[1][0], out[0][0]))
        assert rel(out[1][1], out[0][1]) <= 10 * tol, (prec, rel(out[1][1], out[0][1]))
