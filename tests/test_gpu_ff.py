"""The float-float mode (DAFMM_FF): P2M, M2L (by rotation, Sec. 3.4) and the leaves (P2P, L2P) of
uniform trees in float-float arithmetic (pairs of FP32 numbers, about 48 significand bits),
M2M and L2L in FP64.  Its results must match the oracle FMM on the same tree and order to
the FP64 mode's bounds (relative L2 1e-12 potential, 1e-11 field: rounding only), including
with planted close and coincident pairs across leaf faces; adaptive trees take the FP64 path
(bitwise equal to DAFMM_FP64)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def gpu_eval(ctx, x, q, dom, depth, p, prec, max_leaf=64):
    n = len(q)
    tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=dom,
                          uniform_depth=depth, max_leaf=max_leaf)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree.eval(p, phi, E, precision=prec)
    B.dafmm_sync(ctx.h)
    tree.free()
    return phi.cpu().numpy(), E.cpu().numpy()


def test_ff_config1_against_oracle(ctx):
    """N = 1e4 uniform, depth 3, p = 6: float-float against the oracle at the FP64 bounds."""
    cfg = W.C1
    x, q, dom = W.make(cfg)
    ref_phi, ref_E = O.fmm(x, q, dom, cfg["order"], uniform_depth=cfg["uniform_depth"])
    phi, E = gpu_eval(ctx, x, q, dom, cfg["uniform_depth"], cfg["order"], "ff")
    assert rel(phi, ref_phi) <= 1e-12 and rel(E, ref_E) <= 1e-11, (rel(phi, ref_phi), rel(E, ref_E))


@pytest.mark.parametrize("p", [2, 4, 8, 10])
def test_ff_orders_against_oracle(ctx, p):
    """Orders 2..10 on N = 2e4, depth 4 (several leaves per neighbour list and every M2L level)."""
    x, q = W.uniform(20000, seed=900 + p)
    dom = W.UNIT_CUBE
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=4)
    phi, E = gpu_eval(ctx, x, q, dom, 4, p, "ff")
    assert rel(phi, ref_phi) <= 1e-12 and rel(E, ref_E) <= 1e-11, (p, rel(phi, ref_phi), rel(E, ref_E))


def test_ff_close_and_coincident_pairs(ctx):
    """Pairs planted at 1e-4..1e-3 of the domain (1e-3..1e-2 leaf widths) across leaf faces
    (x = 0.5, y = 0.25) and two coincident particles: the float-float near field holds them to
    the FP64 bounds.  (A float-float offset carries 2^-49 leaf widths, so a pair's difference is
    relative to r accurate to about 2^-49 / r: FP64's bounds hold down to pairs of about 1e-3
    leaf widths; closer pairs keep FP64 accuracy relative to the leaf width only.)"""
    rng = np.random.default_rng(77)
    x, q = W.uniform(6000, seed=78)
    n_pl = 200
    base = rng.random((n_pl, 3))
    base[: n_pl // 2, 0] = 0.5 - 1e-4 * rng.random(n_pl // 2)
    base[n_pl // 2:, 1] = 0.25 - 1e-4 * rng.random(n_pl - n_pl // 2)
    step = 10.0 ** rng.uniform(-4, -3, n_pl)
    other = base.copy()
    other[: n_pl // 2, 0] += step[: n_pl // 2]
    other[n_pl // 2:, 1] += step[n_pl // 2:]
    x = np.vstack([x, base, other, x[:1]])  # the last one coincides with particle 0
    q = np.concatenate([q, rng.uniform(-1, 1, 2 * n_pl), [0.5]])
    dom = W.UNIT_CUBE
    ref_phi, ref_E = O.fmm(x, q, dom, 6, uniform_depth=3)
    phi, E = gpu_eval(ctx, x, q, dom, 3, 6, "ff")
    assert rel(phi, ref_phi) <= 1e-12 and rel(E, ref_E) <= 1e-11, (rel(phi, ref_phi), rel(E, ref_E))


def test_ff_adaptive_is_fp64(ctx):
    """Adaptive trees take the FP64 path in this mode: bitwise equal results."""
    x, q = W.clustered(20000, seed=31, charges="signed")
    p64 = gpu_eval(ctx, x, q, None, -1, 6, "fp64", max_leaf=48)
    pff = gpu_eval(ctx, x, q, None, -1, 6, "ff", max_leaf=48)
    assert np.array_equal(p64[0], pff[0]) and np.array_equal(p64[1], pff[1])
