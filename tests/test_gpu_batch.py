"""Batched solves: forests (many independent problems in one adaptive structure), CUDA-graph
replay and pooled contexts, through the C ABI.

A problem solved inside a forest has the tree it would have alone (its own root cube, the
same split rule), and every box's arithmetic runs over the same lists in the same order, so
its potential and field equal the stand-alone solve bit for bit; the stand-alone adaptive
solve itself is held to the oracle (test_gpu_adaptive), and a few forest members are checked
against the oracle directly here."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_02626_gb300 import binding as B
from paper_2508_02626_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 3.8e-6, "fp32": 3.8e-6}
TOL_E = {"fp64": 1e-11, "mixed": 1e-5, "fp32": 1e-5}


@pytest.fixture(scope="module")
def ctx():
    B.load()
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def members(sizes):
    xs, qs = [], []
    for n, kind, seed in sizes:
        x, q = W.batch_member(n, kind, seed)
        xs.append(x)
        qs.append(q)
    offs = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.int64)
    return xs, qs, offs


def eval_dev(tree, n, p, prec):
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    tree.eval(p, phi, E, precision=prec)
    return phi, E


def standalone(ctx, x, q, s, p, prec):
    t = ctx.build_tree(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), domain=None, uniform_depth=-1,
                       max_leaf=s)
    phi, E = eval_dev(t, len(q), p, prec)
    out = phi.cpu().numpy(), E.cpu().numpy(), t.info()["domain"]
    t.free()
    return out


def small_batch():
    sizes = [(n, kind, 900 + k) for k, (n, kind) in enumerate(
        [(1500, "uniform"), (0, "uniform"), (1, "clustered"), (4000, "clustered"), (2, "uniform"),
         (9000, "clustered"), (700, "uniform"), (12000, "uniform"), (64, "clustered"), (3000, "clustered")])]
    return members(sizes)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_forest_equals_standalone(ctx, prec):
    """Ten problems of 0 to 12,000 particles (empty, single-particle, uniform, clustered) in one
    forest: each member's result equals its stand-alone solve bit for bit."""
    xs, qs, offs = small_batch()
    x, q = np.concatenate(xs), np.concatenate(qs)
    s, p = 32, 6
    f = ctx.build_forest(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), offs, max_leaf=s)
    nt, doms = f.forest()
    assert nt == len(xs)
    phi, E = eval_dev(f, len(q), p, prec)
    B.dafmm_sync(ctx.h)
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    f.free()
    for r in range(len(xs)):
        a, b = offs[r], offs[r + 1]
        if b - a == 0:
            continue
        sphi, sE, sdom = standalone(ctx, xs[r], qs[r], s, p, prec)
        assert np.array_equal(doms[r], sdom), r
        assert np.array_equal(phi[a:b], sphi), (r, prec)
        assert np.array_equal(E[a:b], sE), (r, prec)


def test_forest_members_against_oracle(ctx):
    xs, qs, offs = small_batch()
    x, q = np.concatenate(xs), np.concatenate(qs)
    f = ctx.build_forest(x, q, offs, max_leaf=24)  # host buffers
    _, doms = f.forest()
    for prec in ("fp64", "fp32"):
        phi, E = np.zeros(len(q)), np.zeros((len(q), 3))
        f.eval(8, phi, E, precision=prec)
        for r in (3, 5, 7, 2):
            a, b = offs[r], offs[r + 1]
            ref_phi, ref_E = O.fmm(xs[r], qs[r], O.bounding_cube(xs[r]), 8, max_leaf=24, max_depth=20)
            assert np.array_equal(doms[r], O.bounding_cube(xs[r]))
            assert rel(phi[a:b], ref_phi) <= TOL[prec], (r, prec, rel(phi[a:b], ref_phi))
            assert rel(E[a:b], ref_E) <= TOL_E[prec]
    f.free()


def test_forest_given_domains_and_errors(ctx):
    xs, qs, offs = members([(2000, "uniform", 5), (2500, "uniform", 6)])
    x, q = np.concatenate(xs), np.concatenate(qs)
    doms = np.array([[0, 0, 0, 1.0], [-1, -1, -1, 3.0]])
    f = ctx.build_forest(x, q, offs, domains=doms, max_leaf=16)
    assert np.array_equal(f.forest()[1], doms)
    phi = np.zeros(len(q))
    f.eval(5, phi, None)
    f.free()
    for r in range(2):
        ref, _ = O.fmm(xs[r], qs[r], doms[r], 5, max_leaf=16, max_depth=20)
        assert rel(phi[offs[r]:offs[r + 1]], ref) <= 1e-12
    for bad in ([1, 2000, 4500], [0, 3000, 2000], [0]):
        with pytest.raises(B.DafmmError) as e:
            ctx.build_forest(x, q, np.array(bad), max_leaf=16)
        assert e.value.code == B.DAFMM_ERR_INVALID_ARG


def test_graph_replay_matches_eval(ctx):
    """A forest evaluated by CUDA-graph replay: the same bits as dafmm_eval, replay after
    replay; the graph holds every kernel of the evaluation."""
    xs, qs, offs = small_batch()
    x, q = np.concatenate(xs), np.concatenate(qs)
    f = ctx.build_forest(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), offs, max_leaf=32)
    phi0, E0 = eval_dev(f, len(q), 6, "fp32")
    phi0, E0 = phi0.cpu().numpy(), E0.cpu().numpy()
    phi = torch.zeros(len(q), dtype=torch.float64, device="cuda")
    E = torch.zeros((len(q), 3), dtype=torch.float64, device="cuda")
    g = f.graph(6, phi, E, precision="fp32")
    assert g.nodes() >= 5
    s = torch.cuda.Stream()
    for _ in range(3):
        phi.zero_()
        E.zero_()
        torch.cuda.synchronize()
        g.launch(s)
        s.synchronize()
        assert np.array_equal(phi.cpu().numpy(), phi0) and np.array_equal(E.cpu().numpy(), E0)
    B.dafmm_sync(ctx.h)
    g.free()
    f.free()


def test_pooled_context_reuse():
    """A pooled context: repeated build / evaluate / free cycles return every block to the
    pool and give the same results as an ordinary context."""
    xs, qs, offs = small_batch()
    x, q = np.concatenate(xs), np.concatenate(qs)
    plain = B.Context(0)
    f = plain.build_forest(x, q, offs, max_leaf=32)
    ref = np.zeros(len(q))
    f.eval(6, ref, None, precision="fp32")
    f.free()
    plain.close()
    pool = B.Context(0, pool_bytes=256 << 20)
    base = None
    for it in range(4):
        f = pool.build_forest(x, q, offs, max_leaf=32)
        phi = np.zeros(len(q))
        f.eval(6, phi, None, precision="fp32")
        f.free()
        assert np.array_equal(phi, ref)
        used = B.dafmm_bytes_in_use(pool.h)
        base = used if base is None else base
        assert used == base  # only the per-order tables stay
    # a request larger than the pool fails cleanly and leaves the pool usable
    big, bq = W.uniform(3_000_000, seed=1)
    with pytest.raises(B.DafmmError) as e:
        pool.build_forest(big, bq, [0, len(bq)], max_leaf=32)
    assert e.value.code == B.DAFMM_ERR_OVER_BUDGET
    assert B.dafmm_bytes_in_use(pool.h) == base
    f = pool.build_forest(x, q, offs, max_leaf=32)
    phi = np.zeros(len(q))
    f.eval(6, phi, None, precision="fp32")
    f.free()
    assert np.array_equal(phi, ref)
    pool.close()


def test_batch_256_sampled(ctx):
    """The batched workload: 256 problems, N log-uniform in [1e3, 1e5], uniform or clustered
    by seed, p = 6, one forest evaluated by one graph launch; 8 sampled members equal their
    stand-alone solves bit for bit, 2 are held to the oracle."""
    sizes = W.batch_sizes()
    xs, qs, offs = members(sizes)
    x, q = np.concatenate(xs), np.concatenate(qs)
    f = ctx.build_forest(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), offs, max_leaf=32)
    phi = torch.zeros(len(q), dtype=torch.float64, device="cuda")
    E = torch.zeros((len(q), 3), dtype=torch.float64, device="cuda")
    g = f.graph(6, phi, E, precision="fp32")
    phi.zero_()
    torch.cuda.synchronize()
    g.launch()
    B.dafmm_sync(ctx.h)
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    g.free()
    f.free()
    rng = np.random.default_rng(11)
    for r in rng.choice(len(sizes), 8, replace=False):
        a, b = offs[r], offs[r + 1]
        sphi, sE, _ = standalone(ctx, xs[r], qs[r], 32, 6, "fp32")
        assert np.array_equal(phi[a:b], sphi) and np.array_equal(E[a:b], sE), r
    for r in rng.choice(len(sizes), 2, replace=False):
        a, b = offs[r], offs[r + 1]
        ref_phi, ref_E = O.fmm(xs[r], qs[r], O.bounding_cube(xs[r]), 6, max_leaf=32, max_depth=20)
        assert rel(phi[a:b], ref_phi) <= TOL["fp32"] and rel(E[a:b], ref_E) <= TOL_E["fp32"]


def test_leaf_tile_does_not_change_results(ctx):
    xs, qs, offs = small_batch()
    x, q = np.concatenate(xs), np.concatenate(qs)
    f = ctx.build_forest(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), offs, max_leaf=32)
    outs = []
    try:
        for w in (1, 2, 4, 8):
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, w)
            phi, E = eval_dev(f, len(q), 6, "fp32")
            outs.append((phi.cpu().numpy(), E.cpu().numpy()))
    finally:
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, 4)
    f.free()
    for phi, E in outs[1:]:
        assert np.array_equal(phi, outs[0][0]) and np.array_equal(E, outs[0][1])
    with pytest.raises(B.DafmmError):
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, 3)


def test_autotuner_picks_and_caches(ctx, tmp_path):
    from paper_2508_02626_gb300 import autotune as A
    xs, qs, offs = small_batch()
    x, q = np.concatenate(xs), np.concatenate(qs)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    path = str(tmp_path / "tune.json")
    try:
        r1 = A.tune_forest(ctx, xt, qt, offs, 6, "fp32", cache=A.Cache(path), reps=1)
        assert not r1["cached"]
        assert r1["max_leaf"] in A.leaf_candidates(6) and r1["leaf_warps"] in A.LEAF_WARPS
        assert len(r1["trials"]) == len(A.leaf_candidates(6)) * len(A.LEAF_WARPS)
        assert r1["ms"] == min(t["build_ms"] + t["eval_ms"] for t in r1["trials"])
        r2 = A.tune_forest(ctx, xt, qt, offs, 6, "fp32", cache=A.Cache(path))
        assert r2["cached"] and r2["max_leaf"] == r1["max_leaf"] and r2["leaf_warps"] == r1["leaf_warps"]
    finally:
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, 4)


def test_pooled_uniform_build_from_host_arrays():
    """A pooled context builds a uniform tree from host arrays asynchronously: the call returns
    once the arrays are copied, the rest of the build stays in flight on its stream, and every
    later call on the tree is ordered after it.  Checked against an ordinary context's
    synchronous build, bit for bit: evaluation right after the build on the build's stream, on
    another stream, and through pageable and pinned host outputs; the tree's information
    (largest leaf, read back on demand) right after the build; the host input arrays
    overwritten as soon as the build returns; a tree freed without evaluation; and the pool
    back to its baseline after every cycle."""
    n, depth, p = 60_000, 4, 6
    x, q = W.uniform(n, seed=77)
    dom = W.UNIT_CUBE
    plain = B.Context(0)
    t = plain.build_tree(x, q, domain=dom, uniform_depth=depth)
    info_ref = t.info()
    ref_phi, ref_E = np.zeros(n), np.zeros((n, 3))
    t.eval(p, ref_phi, ref_E, precision="fp32")
    t.free()
    plain.close()
    pool = B.Context(0, pool_bytes=1 << 30)
    side = torch.cuda.Stream()
    xp, qp = torch.from_numpy(x.copy()).pin_memory(), torch.from_numpy(q.copy()).pin_memory()
    php = torch.zeros(n, dtype=torch.float64).pin_memory()
    Ep = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    base = None
    for it in range(4):
        xp.copy_(torch.from_numpy(x))
        qp.copy_(torch.from_numpy(q))
        t = pool.build_tree(xp, qp, domain=dom, uniform_depth=depth, stream=side if it % 2 else None)
        xp.fill_(float("nan"))  # the host arrays are free once the call returns
        qp.fill_(float("nan"))
        if it == 0:
            info = t.info()
            assert all(info[k] == info_ref[k] for k in info_ref if k != "domain"), (info, info_ref)
        if it == 2:  # freed without evaluation
            t.free()
            torch.cuda.synchronize()
            continue
        if it == 3:  # evaluated on another stream than the build's
            other = torch.cuda.Stream()
            phi = np.zeros(n)
            E = np.zeros((n, 3))
            t.eval(p, phi, E, precision="fp32", stream=other)
        else:
            t.eval(p, php, Ep, precision="fp32", stream=side if it % 2 else None)
            phi, E = php.numpy().copy(), Ep.numpy().copy()
        assert np.array_equal(phi, ref_phi), it
        assert np.array_equal(E, ref_E), it
        t.free()
        torch.cuda.synchronize()
        used = B.dafmm_bytes_in_use(pool.h)
        base = used if base is None else base
        assert used == base, (it, used, base)
    pool.close()
