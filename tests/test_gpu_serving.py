"""The serving loop (dafmm_server_*): requests of mixed sizes, orders and distributions,
submitted while others run, are batched and overlapped, and each result equals the
stand-alone adaptive solve of the same request bit for bit (each request keeps its own tree
inside its job's forest; the stand-alone solve is held to the oracle in test_gpu_adaptive)."""
import time

import numpy as np
import pytest
import torch

from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.Context(0)
    yield c
    c.close()


def standalone(ctx, x, q, p, prec, s):
    t = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), uniform_depth=-1, max_leaf=s)
    phi = torch.empty(len(q), dtype=torch.float64, device="cuda")
    E = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
    t.eval(p, phi, E, precision=prec)
    out = phi.cpu().numpy(), E.cpu().numpy()
    t.free()
    return out


def test_mixed_stream_equals_alone(ctx):
    """One large request occupies a slot while 30 small ones arrive: the small ones are
    batched (fewer jobs than requests) and run beside it; then a trickle of requests of
    orders 4, 6 and 8 arrives one by one.  Every result equals its solve alone."""
    rng = np.random.default_rng(5)
    reqs = [(W.uniform(600_000, seed=1), 8)]
    for k in range(30):
        reqs.append((W.batch_member(int(rng.integers(500, 20000)), "clustered" if k % 2 else "uniform", 100 + k), 6))
    for k in range(12):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
        reqs.append((W.batch_member(n, "uniform" if k % 3 else "clustered", 200 + k), int(rng.choice([4, 6, 8]))))
    srv = B.Server(0, pool_bytes=6 << 30, slots=3, max_batch=16)
    ids = []
    for i, ((x, q), p) in enumerate(reqs):
        ids.append(srv.submit(x, q, p, precision="fp32", max_leaf=48))
        if i >= 31:
            time.sleep(0.002)
    outs = [srv.wait(i, timeout=120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert all(o[0] == B.DAFMM_OK for o in outs), [o[0] for o in outs]
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["jobs"] < len(reqs) and st["requests_per_job"] > 1.0
    assert st["peak_running"] >= 2
    for ((x, q), p), (_, phi, E, times) in zip(reqs, outs):
        sphi, sE = standalone(ctx, x, q, p, "fp32", 48)
        assert np.array_equal(phi, sphi) and np.array_equal(E, sE)
        assert times["latency_ms"] >= times["device_ms"] >= 0.0


def test_over_budget_and_recovery():
    """A request larger than the whole pool fails with OVER_BUDGET; the loop keeps serving."""
    srv = B.Server(0, pool_bytes=192 << 20, slots=2, max_batch=4)
    xb, qb = W.uniform(4_000_000, seed=3)
    big = srv.submit(xb, qb, 6)
    xs, qs = W.uniform(5000, seed=4)
    small = srv.submit(xs, qs, 6)
    st_big = srv.wait(big, timeout=120.0)[0]
    st_small, phi, _, _ = srv.wait(small, timeout=120.0)
    stats = srv.stats()
    srv.close()
    assert st_big == B.DAFMM_ERR_OVER_BUDGET
    assert st_small == B.DAFMM_OK and np.all(np.isfinite(phi))
    assert stats["failed"] == 1 and stats["completed"] == 1


def test_wait_timeout_and_errors():
    srv = B.Server(0, pool_bytes=1 << 30, slots=1, max_batch=2)
    x, q = W.uniform(200_000, seed=9)
    a = srv.submit(x, q, 8)
    b = srv.submit(x, q, 8, precision="fp64")
    assert srv.wait(b, timeout=0.0)[0] in (B.DAFMM_ERR_TIMEOUT, B.DAFMM_OK)
    assert srv.wait(a, timeout=120.0)[0] == B.DAFMM_OK
    assert srv.wait(b, timeout=120.0)[0] == B.DAFMM_OK
    with pytest.raises(B.DafmmError):
        srv.submit(x, q, 11)
    srv.close()


def test_two_waiters_and_consumed_ids():
    """Two threads waiting for one request: one receives its status, the other
    DAFMM_ERR_INVALID_ARG (the request is gone once taken); waiting again for a consumed id is
    DAFMM_ERR_INVALID_ARG as well."""
    import threading
    srv = B.Server(0, pool_bytes=1 << 30, slots=1, max_batch=2)
    x, q = W.uniform(200_000, seed=11)
    rid = srv.submit(x, q, 8)
    got = []

    def waiter():
        got.append(B.dafmm_server_wait(srv.h, rid, 120.0)[0])

    ts = [threading.Thread(target=waiter) for _ in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    again = B.dafmm_server_wait(srv.h, rid, 0.0)[0]
    srv._live.pop(rid)  # the raw waits above took the request: release its buffers here
    st, phi, _, _ = srv.wait(rid, timeout=0.0)  # the wrapper reports an id it no longer holds
    srv.close()
    assert sorted(got) == sorted([B.DAFMM_OK, B.DAFMM_ERR_INVALID_ARG])
    assert again == B.DAFMM_ERR_INVALID_ARG and st == B.DAFMM_ERR_INVALID_ARG and phi is None
