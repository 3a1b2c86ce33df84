"""Adaptive trees (Sec. 3.5: a box with more than s particles is split) on the GPU against
the oracle, through the C ABI.

Both sides build the same tree from the same 21-bit box membership and the same split
rule, number the boxes breadth-first in the same order and use the same U/V/W/X lists
(Cheng, Greengard and Rokhlin), so the FP64 GPU result equals the oracle's up to rounding
(relative L2 <= 1e-12 for the potential, 1e-11 for the field), and the tree statistics
(boxes, leaves, finest level, largest leaf, U and V list entries) are equal exactly.  The
MIXED and FP32 paths are held to the bounds derived for the uniform tree: 64 u and 160 u
with u = 2^-24."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 3.8e-6, "fp32": 3.8e-6}
TOL_E = {"fp64": 1e-11, "mixed": 1e-5, "fp32": 1e-5}
MAX_DEPTH = 20  # the GPU tree's deepest level


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def gpu_eval(ctx, x, q, dom, s, p, prec, host=False, info=False):
    n = len(q)
    if host:
        tree = ctx.build_tree(x, q, domain=dom, uniform_depth=-1, max_leaf=s)
        phi, E = np.zeros(n), np.zeros((n, 3))
        tree.eval(p, phi, E, precision=prec)
    else:
        tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=dom, uniform_depth=-1,
                              max_leaf=s)
        phi_t = torch.empty(n, dtype=torch.float64, device="cuda")
        E_t = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        tree.eval(p, phi_t, E_t, precision=prec)
        B.dafmm_sync(ctx.h)
        phi, E = phi_t.cpu().numpy(), E_t.cpu().numpy()
    ti = tree.info()
    tree.free()
    return (phi, E, ti) if info else (phi, E)


def oracle_stats(x, dom, s):
    t = O.Tree(x, dom, uniform_depth=-1, max_leaf=s, max_depth=MAX_DEPTH)
    leaves = np.flatnonzero(t.is_leaf)
    nu = sum(len(t.list(b, "U")) for b in leaves)
    nv = sum(len(t.list(b, "V")) for b in range(t.nbox))
    return dict(boxes=t.nbox, leaves=len(leaves), depth=int(t.level.max()),
                max_per_leaf=int((t.pend - t.pbeg)[leaves].max()) if len(leaves) else 0,
                p2p_leaf_pairs=nu, m2l_pairs=nv)


def check(ctx, x, q, dom, s, p, precs=("fp64", "mixed", "fp32"), stats=True):
    ref_phi, ref_E = O.fmm(x, q, dom, p, max_leaf=s, max_depth=MAX_DEPTH)
    for prec in precs:
        phi, E, ti = gpu_eval(ctx, x, q, dom, s, p, prec, info=True)
        assert rel(phi, ref_phi) <= TOL[prec], (prec, rel(phi, ref_phi))
        assert rel(E, ref_E) <= TOL_E[prec], (prec, rel(E, ref_E))
    if stats:
        assert ti["adaptive"] == 1
        st = oracle_stats(x, dom, s)
        for k, v in st.items():
            assert ti[k] == v, (k, ti[k], v)
    return ref_phi


def test_clustered_20k_s32_p6(ctx):
    """32 Gaussian clusters (the clustered workload's recipe), s = 32: levels 0 to ~7."""
    x, q = W.clustered(20000, seed=21, charges="signed")
    dom = O.bounding_cube(x)
    check(ctx, x, q, dom, 32, 6)


@pytest.mark.parametrize("p", [0, 1, 2, 4, 8, 10])
def test_every_order(ctx, p):
    x, q = W.clustered(6000, seed=400 + p, charges="signed")
    dom = O.bounding_cube(x)
    check(ctx, x, q, dom, 24, p, precs=("fp64", "fp32"), stats=p == 4)


def test_gaussian_blob_and_method_error(ctx):
    """One Gaussian blob (the paper's test distribution, Sec. 3.5), s = 40, p = 8: the FP64
    result's error against the direct sum (Eq. 1) is the oracle's to 1% (the method's own
    truncation error, here ~2.5e-7); the FP32 result's is within that plus its rounding
    bound (triangle inequality)."""
    x, q = W.gaussian(15000, seed=8)
    dom = O.bounding_cube(x)
    ref_phi = check(ctx, x, q, dom, 40, 8, precs=("fp64", "fp32"))
    d_phi, _ = O.direct(x, q)
    sig = rel(ref_phi, d_phi)
    phi, _ = gpu_eval(ctx, x, q, dom, 40, 8, "fp64")
    assert abs(rel(phi, d_phi) / sig - 1.0) < 0.01
    phi, _ = gpu_eval(ctx, x, q, dom, 40, 8, "fp32")
    assert rel(phi, d_phi) <= sig + TOL["fp32"]


def test_deep_tree(ctx):
    """Pairs of particles 1e-5 apart at random positions and s = 1: leaves down to
    level ~17, long chains of single-child boxes, W and X lists across many levels."""
    rng = np.random.default_rng(31)
    c = rng.random((400, 3))
    x = np.vstack([c, c + 1e-5 * rng.standard_normal((400, 3))])
    q = rng.uniform(-1, 1, len(x))
    dom = W.UNIT_CUBE
    check(ctx, x, q, dom, 1, 5)
    _, _, ti = gpu_eval(ctx, x, q, dom, 1, 5, "fp64", info=True)
    assert ti["depth"] >= 14


def test_single_leaf_is_direct_sum(ctx):
    """s >= n: the root is the only leaf and the result is the direct sum (Eq. 1)."""
    x, q = W.clustered(3000, seed=5, charges="signed")
    dom = O.bounding_cube(x)
    d_phi, d_E = O.direct(x, q)
    phi, E, ti = gpu_eval(ctx, x, q, dom, 3000, 6, "fp64", info=True)
    assert ti["boxes"] == 1 and ti["leaves"] == 1
    assert rel(phi, d_phi) <= 1e-13 and rel(E, d_E) <= 1e-12


def test_edge_cases(ctx):
    dom = W.UNIT_CUBE
    # empty input
    tree = ctx.build_tree(np.zeros((0, 3)), np.zeros(0), domain=dom, uniform_depth=-1, max_leaf=8)
    tree.eval(4, np.zeros(0), np.zeros((0, 3)))
    tree.free()
    # coincident points beyond s stop at the deepest level; boundary points; host buffers
    rng = np.random.default_rng(3)
    x = np.vstack([rng.random((2000, 3)), np.tile([[0.25, 0.5, 0.75]], (12, 1)), [[0, 0, 0], [1, 1, 1]]])
    q = rng.uniform(-1, 1, len(x))
    ref_phi, ref_E = O.fmm(x, q, dom, 6, max_leaf=8, max_depth=MAX_DEPTH)
    for host in (False, True):
        phi, E, ti = gpu_eval(ctx, x, q, dom, 8, 6, "fp64", host=host, info=True)
        assert rel(phi, ref_phi) <= 1e-12 and rel(E, ref_E) <= 1e-11
    assert ti["depth"] == MAX_DEPTH and ti["max_per_leaf"] >= 12
    # invalid s
    with pytest.raises(B.DafmmError) as e:
        ctx.build_tree(x, q, domain=dom, uniform_depth=-1, max_leaf=0)
    assert e.value.code == B.DAFMM_ERR_INVALID_ARG


def test_reuse_across_orders_and_precisions(ctx):
    """One tree evaluated at several orders and precisions in turn: every result equals a
    fresh tree's, bit for bit."""
    x, q = W.clustered(8000, seed=17, charges="signed")
    dom = O.bounding_cube(x)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    tree = ctx.build_tree(xt, qt, domain=dom, uniform_depth=-1, max_leaf=32)
    outs = {}
    for p, prec in ((6, "fp32"), (8, "fp64"), (6, "fp32"), (6, "mixed")):
        phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
        tree.eval(p, phi, None, precision=prec)
        outs.setdefault((p, prec), []).append(phi.cpu().numpy())
    tree.free()
    assert np.array_equal(outs[(6, "fp32")][0], outs[(6, "fp32")][1])
    fresh, _ = gpu_eval(ctx, x, q, dom, 32, 8, "fp64")
    assert np.array_equal(fresh, outs[(8, "fp64")][0])


def test_clustered_4e6_p10_sampled(ctx):
    """N = 4,000,000 in 32 clusters, s = 64, p = 10 (the adaptive benchmark workload): FP64
    and FP32 against the oracle FMM on 100 sampled targets."""
    cfg = W.C3
    x, q, _ = W.make(cfg)
    dom = O.bounding_cube(x)
    rng = np.random.default_rng(79)
    tg = np.sort(rng.choice(cfg["n"], 100, replace=False))
    ref_phi, ref_E = O.fmm(x, q, dom, cfg["order"], max_leaf=cfg["max_leaf"], max_depth=MAX_DEPTH, targets=tg)
    for prec in ("fp64", "fp32"):
        phi, E = gpu_eval(ctx, x, q, dom, cfg["max_leaf"], cfg["order"], prec)
        assert rel(phi[tg], ref_phi) <= TOL[prec], (prec, rel(phi[tg], ref_phi))
        assert rel(E[tg], ref_E) <= TOL_E[prec], (prec, rel(E[tg], ref_E))


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, 9, 10])
def test_tensor_core_gathered_m2l(ctx, p):
    """The gathered tcgen05 M2L (TF32 split products, sources gathered row by row) against the
    SIMT FP32 M2L and the oracle, on a clustered tree with levels 2 to ~8 and partial tiles;
    p = 9, 10 split the output columns in two halves."""
    x, q = W.clustered(12000, seed=500 + p, charges="signed")
    dom = O.bounding_cube(x)
    ref_phi, ref_E = O.fmm(x, q, dom, p, max_leaf=20, max_depth=MAX_DEPTH)
    for prec in ("mixed", "fp32"):
        tc_phi, tc_E = gpu_eval(ctx, x, q, dom, 20, p, prec)
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_KERNEL, 1)
        try:
            si_phi, si_E = gpu_eval(ctx, x, q, dom, 20, p, prec)
        finally:
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_KERNEL, 0)
        assert rel(tc_phi, ref_phi) <= TOL[prec], (prec, rel(tc_phi, ref_phi))
        assert rel(tc_E, ref_E) <= TOL_E[prec], (prec, rel(tc_E, ref_E))
        assert rel(si_phi, ref_phi) <= TOL[prec]
        assert rel(tc_phi, si_phi) <= TOL[prec]


@pytest.mark.parametrize("p", [4, 8, 10])
def test_gathered_m2l_operand_splits(ctx, p):
    """The gathered M2L with F16 and with TF32 split operands (FP32 mode), clustered tree."""
    x, q = W.clustered(12000, seed=600 + p, charges="signed")
    dom = O.bounding_cube(x)
    ref_phi, ref_E = O.fmm(x, q, dom, p, max_leaf=20, max_depth=MAX_DEPTH)
    for f16 in (1, 0):
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_F16, f16)
        try:
            phi, E = gpu_eval(ctx, x, q, dom, 20, p, "fp32")
        finally:
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_F16, 1)
        assert rel(phi, ref_phi) <= TOL["fp32"], (f16, rel(phi, ref_phi))
        assert rel(E, ref_E) <= TOL_E["fp32"]


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10])
def test_gathered_m2l_harmonic(ctx, p):
    """The gathered M2L in the harmonic basis (the default: the (p + 1)^2 free coefficients
    gathered and contracted, the others restored by Laplace's equation) and in the full basis,
    FP32 mode (F16 operands) and MIXED (TF32 operands), on a clustered tree with levels 2 to ~8:
    both within the mode's bound of the oracle and of each other."""
    x, q = W.clustered(12000, seed=650 + p, charges="signed")
    dom = O.bounding_cube(x)
    ref_phi, ref_E = O.fmm(x, q, dom, p, max_leaf=20, max_depth=MAX_DEPTH)
    for prec in ("fp32", "mixed"):
        out = {}
        for harm in (1, 0):
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, harm)
            try:
                out[harm] = gpu_eval(ctx, x, q, dom, 20, p, prec)
            finally:
                B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, 1)
            assert rel(out[harm][0], ref_phi) <= TOL[prec], (prec, harm, rel(out[harm][0], ref_phi))
            assert rel(out[harm][1], ref_E) <= TOL_E[prec], (prec, harm, rel(out[harm][1], ref_E))
        assert rel(out[1][0], out[0][0]) <= TOL[prec]
