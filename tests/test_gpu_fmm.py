"""Whole-FMM parity of the GPU path with the oracle, through the C ABI.

The oracle runs the same traversal (Sec. 1) on the same tree with the same order, so
the FP64 GPU result must equal it up to rounding: relative L2 <= 1e-12 (potential and
field).  The MIXED and FP32 paths compute P2M, M2L, L2P and P2P in FP32 (unit roundoff
u = 2^-24 ~ 6e-8): every coefficient and pair term carries a few u, and the sums over
~10^2-10^4 partially cancelling terms amplify that, so they are held to 64 u ~ 3.8e-6 for
the potential and 160 u ~ 1e-5 for the field (measured: 5e-7 to 8e-7 and 1e-6 to 3e-6).
Against the direct sum (Eq. 1) every path carries the method's own truncation error,
which must match the oracle's to 1%."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 3.8e-6, "fp32": 3.8e-6}
TOL_E = {"fp64": 1e-11, "mixed": 1e-5, "fp32": 1e-5}
PT_TOL = 512 * 2.0 ** -24  # worst single target, relative to max(|value|, median |value|)


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def gpu_eval(ctx, x, q, dom, depth, p, prec, host=False):
    n = len(q)
    if host:
        tree = ctx.build_tree(x, q, domain=dom, uniform_depth=depth)
        phi, E = np.zeros(n), np.zeros((n, 3))
        tree.eval(p, phi, E, precision=prec)
        tree.free()
        return phi, E
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    tree = ctx.build_tree(xt, qt, domain=dom, uniform_depth=depth)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree.eval(p, phi, E, precision=prec)
    B.dafmm_sync(ctx.h)  # raises if a bounded device wait gave up
    tree.free()
    return phi.cpu().numpy(), E.cpu().numpy()


def test_config1_uniform_1e4_p6(ctx):
    """N=10,000 uniform in the unit cube, q in [-1,1], depth 3, p=6, all targets."""
    cfg = W.C1
    x, q, dom = W.make(cfg)
    ref_phi, ref_E = O.fmm(x, q, dom, cfg["order"], uniform_depth=cfg["uniform_depth"])
    d_phi, d_E = O.direct(x, q)
    sig_oracle = rel(ref_phi, d_phi)
    for prec in ("fp64", "mixed", "fp32"):
        phi, E = gpu_eval(ctx, x, q, dom, cfg["uniform_depth"], cfg["order"], prec)
        assert rel(phi, ref_phi) <= TOL[prec], (prec, rel(phi, ref_phi))
        assert rel(E, ref_E) <= TOL_E[prec], (prec, rel(E, ref_E))
        assert abs(rel(phi, d_phi) / sig_oracle - 1.0) < 0.01


@pytest.mark.parametrize("p", [0, 1, 2, 3, 5, 7, 9, 10])
def test_every_order_fp64(ctx, p):
    x, q = W.uniform(3000, seed=77 + p)
    dom = W.UNIT_CUBE
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=3)
    phi, E = gpu_eval(ctx, x, q, dom, 3, p, "fp64")
    assert rel(phi, ref_phi) <= 1e-12 and rel(E, ref_E) <= 1e-11


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, 9, 10])
def test_tensor_core_m2l(ctx, p):
    """The tcgen05 contractions (TF32 split products) against the oracle: M2L alone (MIXED)
    and against the SIMT FP32 M2L, and M2L + M2M + L2L (FP32 mode), on a depth-4 tree
    (levels 2-4: tiles of 8, 64 and 128 boxes); p = 9, 10 split N in two."""
    x, q = W.uniform(20000, seed=300 + p)
    dom = W.UNIT_CUBE
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=4)
    tc_phi, tc_E = gpu_eval(ctx, x, q, dom, 4, p, "mixed")
    B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_KERNEL, 1)
    try:
        si_phi, si_E = gpu_eval(ctx, x, q, dom, 4, p, "mixed")
    finally:
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_KERNEL, 0)
    assert rel(tc_phi, ref_phi) <= TOL["mixed"], rel(tc_phi, ref_phi)
    assert rel(tc_E, ref_E) <= TOL_E["mixed"]
    assert rel(si_phi, ref_phi) <= TOL["mixed"]
    assert rel(tc_phi, si_phi) <= TOL["mixed"]
    # FP32 mode: L2L on the tensor cores as well (the default), and M2M too (mask 7)
    for mask in (5, 7):
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_TC_MASK, mask)
        try:
            f_phi, f_E = gpu_eval(ctx, x, q, dom, 4, p, "fp32")
        finally:
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_TC_MASK, 5)
        assert rel(f_phi, ref_phi) <= TOL["fp32"], (mask, rel(f_phi, ref_phi))
        assert rel(f_E, ref_E) <= TOL_E["fp32"]


@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_depths_and_near_field(ctx, depth):
    x, q = W.uniform(6000 if depth < 4 else 30000, seed=50 + depth)
    dom = W.UNIT_CUBE
    p = 5
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=depth)
    for prec in ("fp64", "mixed"):
        phi, E = gpu_eval(ctx, x, q, dom, depth, p, prec)
        assert rel(phi, ref_phi) <= TOL[prec] and rel(E, ref_E) <= TOL_E[prec]
    if depth <= 1:  # no far field: equals the direct sum
        d_phi, d_E = O.direct(x, q)
        phi, E = gpu_eval(ctx, x, q, dom, depth, p, "fp64")
        assert rel(phi, d_phi) <= 1e-13 and rel(E, d_E) <= 1e-12


def test_edge_cases(ctx):
    dom = W.UNIT_CUBE
    # empty input
    tree = ctx.build_tree(np.zeros((0, 3)), np.zeros(0), domain=dom, uniform_depth=3)
    tree.eval(4, np.zeros(0), np.zeros((0, 3)))
    tree.free()
    # one particle: no partner, zero potential
    phi, E = gpu_eval(ctx, np.array([[0.3, 0.3, 0.3]]), np.array([1.0]), dom, 2, 4, "fp64", host=True)
    assert phi[0] == 0.0 and np.all(E == 0.0)
    # boundary points (x = 0 and x = 1 exactly, clamped into the last box), coincident
    # points, clustered data leaving most leaves empty, host buffers
    rng = np.random.default_rng(9)
    x = np.vstack([rng.random((1500, 3)) * 0.2, [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.1, 0.1, 0.1], [0.1, 0.1, 0.1]]])
    q = rng.uniform(-1, 1, len(x))
    for p in (3, 6):
        ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=4)
        for host in (False, True):
            phi, E = gpu_eval(ctx, x, q, dom, 4, p, "fp64", host=host)
            assert rel(phi, ref_phi) <= 1e-12 and rel(E, ref_E) <= 1e-11


def test_bounding_cube_domain(ctx):
    x, q = W.clustered(4000, seed=12)
    tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=None, uniform_depth=3)
    dom = tree.info()["domain"]
    assert np.array_equal(dom, O.bounding_cube(x))
    phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
    E = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
    tree.eval(6, phi, E)
    torch.cuda.synchronize()
    tree.free()
    ref_phi, ref_E = O.fmm(x, q, dom, 6, uniform_depth=3)
    assert rel(phi.cpu().numpy(), ref_phi) <= 1e-12 and rel(E.cpu().numpy(), ref_E) <= 1e-11


def test_deterministic_and_reusable(ctx):
    x, q = W.uniform(20000, seed=5)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    tree = ctx.build_tree(xt, qt, domain=W.UNIT_CUBE, uniform_depth=4)
    outs = []
    for prec in ("mixed", "mixed", "fp64", "mixed"):
        phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
        tree.eval(6, phi, None, precision=prec)
        outs.append(phi.cpu().numpy())
    tree.free()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[3])


def test_errors_are_codes(ctx):
    x, q = W.uniform(100, seed=1)
    tree = ctx.build_tree(x, q, domain=W.UNIT_CUBE, uniform_depth=2)
    for kw, code in ((dict(order=11), B.DAFMM_ERR_UNSUPPORTED_ORDER),
                     (dict(order=4, theta=0.5), B.DAFMM_ERR_UNSUPPORTED)):
        with pytest.raises(B.DafmmError) as e:
            tree.eval(phi=np.zeros(100), **kw)
        assert e.value.code == code
    tree.free()
    small = B.Context(0, hbm_budget_bytes=4096)
    with pytest.raises(B.DafmmError) as e:
        small.build_tree(x, q, domain=W.UNIT_CUBE, uniform_depth=2)
    assert e.value.code == B.DAFMM_ERR_OVER_BUDGET
    small.close()
    with pytest.raises(B.DafmmError) as e:
        ctx.build_tree(x, q, domain=[0, 0, 0, -1.0], uniform_depth=2)
    assert e.value.code == B.DAFMM_ERR_INVALID_ARG


def test_config2_full_size_sampled(ctx):
    """N=1,000,000 uniform, depth 5, p=8 (the benchmark workload, same launch path):
    FP64 and MIXED against the oracle FMM on 200 sampled targets."""
    cfg = W.C2
    x, q, dom = W.make(cfg)
    rng = np.random.default_rng(77)
    tg = np.sort(rng.choice(cfg["n"], 200, replace=False))
    ref_phi, ref_E = O.fmm(x, q, dom, cfg["order"], uniform_depth=cfg["uniform_depth"], targets=tg)
    for prec in ("fp64", "mixed"):
        phi, E = gpu_eval(ctx, x, q, dom, cfg["uniform_depth"], cfg["order"], prec)
        assert rel(phi[tg], ref_phi) <= TOL[prec], (prec, rel(phi[tg], ref_phi))
        assert rel(E[tg], ref_E) <= TOL_E[prec], (prec, rel(E[tg], ref_E))


def per_target(a, b):
    """Largest per-target error |a_i - b_i| relative to max(|b_i|, median |b|) (rows are
    vectors for the field): relative where the value is typical or large -- the closest
    pairs give the largest fields -- and relative to a typical value where it cancels to
    near zero, where a relative error has no meaning."""
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    d = np.linalg.norm(a - b, axis=1)
    m = np.linalg.norm(b, axis=1)
    return float((d / np.maximum(m, np.median(m))).max())


def test_config2_full_size_all_particles(ctx):
    """N=1,000,000 uniform, depth 5, p=8 (the benchmark workload): the FP32 mode (the
    benchmark's) and the MIXED mode against a full oracle solve over every particle, so
    that the closest pairs -- whose fields dominate the relative L2 of E -- are all in the
    comparison: relative L2 of the potential and the field within the FP32 bounds, and the
    worst single target within PT_TOL of max(|value|, median |value|)."""
    cfg = W.C2
    x, q, dom = W.make(cfg)
    ref_phi, ref_E = O.fmm(x, q, dom, cfg["order"], uniform_depth=cfg["uniform_depth"])
    for prec in ("fp32", "mixed"):
        phi, E = gpu_eval(ctx, x, q, dom, cfg["uniform_depth"], cfg["order"], prec)
        ep, eE = rel(phi, ref_phi), rel(E, ref_E)
        tp, tE = per_target(phi, ref_phi), per_target(E, ref_E)
        print("%s: rel L2 phi %.3e E %.3e, worst target phi %.3e E %.3e" % (prec, ep, eE, tp, tE))
        assert ep <= TOL[prec] and eE <= TOL_E[prec], (prec, ep, eE)
        assert tp <= PT_TOL and tE <= PT_TOL, (prec, tp, tE)


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10])
def test_m2l_operand_splits(ctx, p):
    """FP32 mode with the M2L operands split into F16 halves (power-of-two scales per box,
    matrix row and matrix; the default) and into TF32 halves: both within the FP32 bound of
    the oracle, and within it of each other."""
    x, q = W.uniform(20000, seed=700 + p)
    dom = W.UNIT_CUBE
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=4)
    out = {}
    for f16 in (1, 0):
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_F16, f16)
        try:
            out[f16] = gpu_eval(ctx, x, q, dom, 4, p, "fp32")
        finally:
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_F16, 1)
        assert rel(out[f16][0], ref_phi) <= TOL["fp32"], (f16, rel(out[f16][0], ref_phi))
        assert rel(out[f16][1], ref_E) <= TOL_E["fp32"]
    assert rel(out[1][0], out[0][0]) <= TOL["fp32"]


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8, 9, 10])
def test_harmonic_m2l(ctx, p):
    """The tensor-core M2L in the harmonic basis (the default: the (p + 1)^2 free coefficients
    contracted, the others restored by Laplace's equation) and in the full basis, FP32 mode (F16
    operands) and MIXED (TF32 operands): both within the mode's bound of the oracle and within it
    of each other; depth 5 at p = 2 and depth 4 otherwise, so that every level and tile shape of
    the kernel runs, and in the FP32 mode with the tensor-core L2L reading level 2's expanded
    locals."""
    depth = 5 if p == 2 else 4
    x, q = W.uniform(30000, seed=800 + p)
    dom = W.UNIT_CUBE
    ref_phi, ref_E = O.fmm(x, q, dom, p, uniform_depth=depth)
    for prec in ("fp32", "mixed"):
        out = {}
        for harm in (1, 0):
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, harm)
            try:
                out[harm] = gpu_eval(ctx, x, q, dom, depth, p, prec)
            finally:
                B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, 1)
            assert rel(out[harm][0], ref_phi) <= TOL[prec], (prec, harm, rel(out[harm][0], ref_phi))
            assert rel(out[harm][1], ref_E) <= TOL_E[prec], (prec, harm, rel(out[harm][1], ref_E))
        assert rel(out[1][0], out[0][0]) <= TOL[prec]
        assert rel(out[1][1], out[0][1]) <= TOL_E[prec]


@pytest.mark.parametrize("p", [3, 6, 8, 10])
def test_harmonic_multipoles(ctx, p):
    """P2M and M2M in the harmonic basis (uniform trees, FP32 and MIXED, the default): the
    multipoles of every level against the oracle's P2M (Eq. 2) of each box's particles about the
    box centre, in box-scaled variables (M~_a = M_a / h^|a|), degree by degree.  The free
    coefficients (z exponent <= 1) are what the device computes: within the FP32 bound.  The
    others are filled in by Laplace's equation on reading; the recursion
    a_i = w1 a_i1 + w2 a_i2 carries the free coefficients' errors into them with gain at most
    G_i = |w1| G_i1 + |w2| G_i2 (G = 1 on the free ones), so they are held to G_i times the bound.
    With the harmonic basis off, every coefficient is within the bound."""
    depth = 4
    x, q = W.uniform(20000, seed=900 + p)
    dom = W.UNIT_CUBE
    ex = O.exponents(p)
    deg = ex.sum(1)
    nc = O.ncoef(p)
    ncp = (nc + 7) // 8 * 8
    idx = {tuple(int(v) for v in e): i for i, e in enumerate(ex)}
    gain = np.ones(nc)
    for i in sorted(range(nc), key=lambda i: ex[i][2]):
        a, b, c = (int(v) for v in ex[i])
        if c >= 2:
            gain[i] = ((a + 2) * (a + 1) * gain[idx[(a + 2, b, c - 2)]] +
                       (b + 2) * (b + 1) * gain[idx[(a, b + 2, c - 2)]]) / (c * (c - 1))
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    n = len(q)
    ref = {}
    for lev in range(2, depth + 1):
        h = dom[3] / 2 ** lev
        ijk = np.minimum(np.floor((x - dom[:3]) / h).astype(int), 2 ** lev - 1)
        P2 = 2 ** (lev - 1)
        oct_ = (ijk[:, 0] & 1) | ((ijk[:, 1] & 1) << 1) | ((ijk[:, 2] & 1) << 2)
        row = oct_ * P2 ** 3 + ((ijk[:, 2] >> 1) * P2 + (ijk[:, 1] >> 1)) * P2 + (ijk[:, 0] >> 1)
        R = np.zeros((8 ** lev, nc))
        for b in np.unique(row):
            sel = row == b
            c = dom[:3] + (ijk[sel][0] + 0.5) * h
            R[b] = O.p2m(p, (x[sel] - c) / h, q[sel])
        ref[lev] = R
    for prec, tol in (("fp32", 2e-5), ("mixed", 2e-5)):
        for harm in (1, 0):
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, harm)
            try:
                tree = ctx.build_tree(xt, qt, domain=dom, uniform_depth=depth)
                phi = torch.empty(n, dtype=torch.float64, device="cuda")
                E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
                tree.eval(p, phi, E, precision=prec)
                B.dafmm_sync(ctx.h)
                for lev in range(2, depth + 1):
                    M = B.dafmm_debug_level(tree.h, "M", lev, ncp)[:, :nc]
                    for k in range(p + 1):
                        s = deg == k
                        scale = np.abs(ref[lev][:, s]).max()
                        err = np.abs(M[:, s] - ref[lev][:, s]).max(0) / scale
                        bound = tol * (gain[s] if harm else 1.0)
                        assert np.all(err <= bound), (prec, harm, lev, k, (err / bound).max())
                tree.free()
            finally:
                B.dafmm_set_option(ctx.h, B.DAFMM_OPT_M2L_HARMONIC, 1)
