"""The allocation-free evaluation entry point (dafmm_eval_noalloc).

It exists for callers that must not allocate device memory while they evaluate (their
memory is owned by their own pool allocator, or cudaMalloc's implicit synchronisation is
not acceptable in their loop).  It keeps every intermediate array in one fixed array of
device memory inside the library; this test checks, through the C ABI, that two calls in
a row give the same potential and field as the ordinary FP64 evaluation (within the FP64
bound of the other parity tests) -- on a depth-3 tree and on the largest accepted case,
order 6 at depth 4, which fills most of the array -- that neither the context's own
allocations nor the device's free memory change across a call, and that requests beyond
its limits are refused.  The file is named so that pytest collects it last."""
import numpy as np
import pytest
import torch

from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def check_twice(ctx, n, p, depth, seed):
    """Two calls in a row against dafmm_eval FP64 on the same tree; returns the tree."""
    x, q = W.uniform(n, seed=seed)
    tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=W.UNIT_CUBE,
                          uniform_depth=depth)
    ref_phi = torch.empty(n, dtype=torch.float64, device="cuda")
    ref_E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree.eval(p, ref_phi, ref_E, precision="fp64")
    B.dafmm_sync(ctx.h)
    ref_phi, ref_E = ref_phi.cpu().numpy(), ref_E.cpu().numpy()
    held = B.dafmm_bytes_in_use(ctx.h)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    for call in range(2):
        phi.fill_(float("nan"))
        E.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        B.dafmm_eval_noalloc(ctx.h, tree.h, p, phi, E)
        B.dafmm_sync(ctx.h)
        free_after = torch.cuda.mem_get_info()[0]
        assert rel(phi.cpu().numpy(), ref_phi) <= 1e-12
        assert rel(E.cpu().numpy(), ref_E) <= 1e-11
        assert B.dafmm_bytes_in_use(ctx.h) == held
        if call == 1:  # the first call on a device may load the library's module
            assert free_after == free_before, (free_before, free_after)
    return tree


def test_noalloc_matches_eval_twice():
    B.load()
    ctx = B.Context(0)
    try:
        n, p = 10_000, 6
        tree = check_twice(ctx, n, p, 3, 1001)
        phi = torch.empty(n, dtype=torch.float64, device="cuda")
        E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        # beyond the limits: order above 6, host outputs
        with pytest.raises(B.DafmmError) as e:
            B.dafmm_eval_noalloc(ctx.h, tree.h, 8, phi, E)
        assert e.value.code == B.DAFMM_ERR_UNSUPPORTED_ORDER
        with pytest.raises(B.DafmmError) as e:
            B.dafmm_eval_noalloc(ctx.h, tree.h, p, np.zeros(n), None)
        assert e.value.code == B.DAFMM_ERR_INVALID_ARG
        tree.free()
        # a tree deeper than 4 levels
        x2, q2 = W.uniform(40_000, seed=3)
        deep = ctx.build_tree(torch.from_numpy(x2).cuda(), torch.from_numpy(q2).cuda(), domain=W.UNIT_CUBE,
                              uniform_depth=5)
        with pytest.raises(B.DafmmError) as e:
            B.dafmm_eval_noalloc(ctx.h, deep.h, 4, torch.empty(40_000, dtype=torch.float64, device="cuda"), None)
        assert e.value.code == B.DAFMM_ERR_INVALID_ARG
        deep.free()
    finally:
        ctx.close()


def test_noalloc_largest_case():
    """Order 6 on a depth-4 tree: the largest case the array accepts (the M2L matrices and
    the expansions of levels 2..4 take about 27 of its 32 MiB)."""
    B.load()
    ctx = B.Context(0)
    try:
        check_twice(ctx, 40_000, 6, 4, 4004).free()
    finally:
        ctx.close()
