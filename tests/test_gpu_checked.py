"""The checked build (libdafmm_check.so, compiled with -DDAFMM_CHECK): every device access whose
index is read from memory is guarded by a check that records a site code, the index and the
bound, and skips the access -- no trap.

On valid inputs no check may fire: tree builds and evaluations of every kind (uniform and
adaptive trees, a forest; FP64 with the rotation M2L, MIXED and FP32 with the tensor-core and
the gathered tensor-core M2L, float-float) return DAFMM_OK from dafmm_sync and hold the oracle
at the same bounds as the unchecked library.  One deliberate failure (dafmm_debug_check: index
32 against the bound 32, into an array of 64) reaches the host as DAFMM_ERR_CHECK naming its
site, index and bound; reading it clears it, and the context keeps working.  The unchecked
library refuses dafmm_debug_check (DAFMM_ERR_UNSUPPORTED)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 3.8e-6, "fp32": 3.8e-6, "ff": 1e-12}
TOL_E = {"fp64": 1e-11, "mixed": 1e-5, "fp32": 1e-5, "ff": 1e-11}


@pytest.fixture(scope="module")
def ctx():
    lib = B.load_checked()
    old = B.swap_library(lib)
    try:
        c = B.Context(0)
        yield c
        c.close()
    finally:
        B.swap_library(old)


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def solve(ctx, x, q, dom, depth, s, p, prec):
    """Build, evaluate and sync through the checked library (dafmm_sync raises on a check)."""
    n = len(q)
    tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=dom,
                          uniform_depth=depth, max_leaf=s)
    B.dafmm_sync(ctx.h)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree.eval(p, phi, E, precision=prec)
    B.dafmm_sync(ctx.h)
    tree.free()
    return phi.cpu().numpy(), E.cpu().numpy()


def test_deliberate_failure_is_reported_and_cleared(ctx):
    B.dafmm_debug_check(ctx.h)
    with pytest.raises(B.DafmmError) as e:
        B.dafmm_sync(ctx.h)
    assert e.value.code == B.DAFMM_ERR_CHECK
    msg = str(e.value)
    assert "site 99" in msg and "index 32" in msg and "bound 32" in msg, msg
    B.dafmm_sync(ctx.h)  # cleared on reading


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32", "ff"])
def test_uniform_runs_clean(ctx, prec):
    """N = 1e4, depth 3, p = 6 in every precision mode: no check fires; oracle bounds hold."""
    cfg = W.C1
    x, q, dom = W.make(cfg)
    ref_phi, ref_E = O.fmm(x, q, dom, cfg["order"], uniform_depth=cfg["uniform_depth"])
    phi, E = solve(ctx, x, q, dom, cfg["uniform_depth"], 64, cfg["order"], prec)
    assert rel(phi, ref_phi) <= TOL[prec] and rel(E, ref_E) <= TOL_E[prec], (prec, rel(phi, ref_phi), rel(E, ref_E))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_adaptive_runs_clean(ctx, prec):
    """A clustered adaptive tree (levels 2 to ~8, U/W/X lists, gathered tensor-core M2L in MIXED
    and FP32, rotation M2L in FP64) at p = 8: no check fires; oracle bounds hold."""
    x, q = W.clustered(12000, seed=4242, charges="signed")
    dom = O.bounding_cube(x)
    ref_phi, ref_E = O.fmm(x, q, dom, 8, max_leaf=20, max_depth=20)
    phi, E = solve(ctx, x, q, dom, -1, 20, 8, prec)
    assert rel(phi, ref_phi) <= TOL[prec] and rel(E, ref_E) <= TOL_E[prec], (prec, rel(phi, ref_phi), rel(E, ref_E))


def test_forest_runs_clean(ctx):
    """A forest of eight problems (empty, one- and two-particle members included), FP32."""
    xs, qs = [], []
    for k, (n, kind) in enumerate([(1500, "uniform"), (0, "uniform"), (1, "clustered"), (4000, "clustered"),
                                   (2, "uniform"), (9000, "clustered"), (700, "uniform"), (64, "clustered")]):
        x, q = W.batch_member(n, kind, 1300 + k)
        xs.append(x)
        qs.append(q)
    offs = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.int64)
    x, q = np.concatenate(xs), np.concatenate(qs)
    f = ctx.build_forest(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), offs, max_leaf=24)
    B.dafmm_sync(ctx.h)
    n = len(q)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    f.eval(6, phi, E, precision="fp32")
    B.dafmm_sync(ctx.h)
    phi = phi.cpu().numpy()
    f.free()
    r = 3  # the 4000-particle clustered member against the oracle on its own cube
    ref, _ = O.fmm(xs[r], qs[r], O.bounding_cube(xs[r]), 6, max_leaf=24, max_depth=20)
    assert rel(phi[offs[r]:offs[r + 1]], ref) <= TOL["fp32"]


def test_unchecked_library_refuses_debug_check():
    lib = B.swap_library(None)  # the checked library, when the fixture holds it
    try:
        c = B.Context(0)
        try:
            with pytest.raises(B.DafmmError) as e:
                B.dafmm_debug_check(c.h)
            assert e.value.code == B.DAFMM_ERR_UNSUPPORTED
        finally:
            c.close()
    finally:
        B.swap_library(lib)
