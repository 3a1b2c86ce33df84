"""Failure detection without a fault: a bounded device wait that runs out reaches the host as
DAFMM_ERR_TIMEOUT through dafmm_sync, and the context keeps working.

dafmm_debug_expire_wait launches one kernel whose mbarrier wait -- the wait of the tensor-core
kernels, bounded by 1 s of device time -- waits for an arrival that nothing makes.  The test
checks the status the host reads, that the record is cleared by reading it, and that the
evaluations before and after (FP32 mode: tensor-core M2M/M2L/L2L with the same waits) are
bitwise equal."""
import time

import numpy as np
import pytest
import torch

from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_context_stays_usable():
    B.load()
    ctx = B.Context(0)
    try:
        x, q = W.uniform(20_000, 7007)
        tree = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(),
                              domain=np.array([0.0, 0.0, 0.0, 1.0]), uniform_depth=3)
        s = torch.cuda.Stream()

        def solve():
            phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
            E = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
            tree.eval(6, phi, E, precision=B.DAFMM_FP32, stream=s)
            B.dafmm_sync(ctx.h, s)  # raises if a wait gave up
            return phi.cpu(), E.cpu()

        phi0, E0 = solve()
        t0 = time.monotonic()
        B.dafmm_debug_expire_wait(ctx.h, s)
        with pytest.raises(B.DafmmError) as err:
            B.dafmm_sync(ctx.h, s)
        waited = time.monotonic() - t0
        assert err.value.code == B.DAFMM_ERR_TIMEOUT
        assert "site 90" in str(err.value)
        # the wait gives up after about 1 s of device time (or 2^26 polls, if sooner)
        assert waited < 30.0
        B.dafmm_sync(ctx.h, s)  # reading the record cleared it
        phi1, E1 = solve()
        assert torch.equal(phi0, phi1) and torch.equal(E0, E1)
        assert torch.isfinite(phi1).all()
        tree.free()
    finally:
        ctx.close()


def test_expire_wait_needs_a_context():
    B.load()
    assert B.load().dafmm_debug_expire_wait(None, None) == B.DAFMM_ERR_INVALID_ARG
