"""Leaf size and near-field tile of adaptive solves, chosen by measurement.

The leaf size s (a box with more than s particles is split, Sec. 3.5) trades near-field work
(P2P over U lists, growing with s) against far-field work (more boxes, more M2L).  The paper
sweeps s on its CPU and tabulates the fastest value per order and particle count (Sec. 3.5,
Table 10: 64 at p = 2, 128 at p = 4, 256 at p = 6 and 8, 512 at p = 10 for large N).
On the GPU the balance is different -- P2P runs at FP32 ALU rate, M2L on the tensor or SIMT
pipes -- so the tuner times candidate values around the paper's choice on the actual
workload (a forest of the problems to solve) together with the near-field kernel's tile
(leaves per thread block, DAFMM_OPT_LEAF_WARPS), and caches the winner as JSON keyed by the
GPU, order, precision and a size class of the workload.
"""
import json
import math
import os
import tempfile
import time

import numpy as np

from . import binding as B

# fastest leaf size of the paper's CPU sweep for large N, per order (Table 10)
PAPER_LEAF_SIZE = {2: 64, 4: 128, 6: 256, 8: 256, 10: 512}
LEAF_WARPS = (2, 4, 8)


def paper_leaf_size(order):
    """The paper's leaf size for `order` (odd orders take the next even order's value)."""
    o = min(10, max(2, order + (order & 1)))
    return PAPER_LEAF_SIZE[o]


def leaf_candidates(order):
    """Powers-of-two fractions of the paper's choice, from s/32 to s (at least 8): the GPU
    favours smaller leaves than the CPU because M2L runs far faster relative to P2P."""
    s0 = paper_leaf_size(order)
    return sorted({max(8, s0 >> k) for k in range(6)})


def size_class(n_total, n_trees):
    """Workloads whose particle count and mean problem size agree within a factor of 2."""
    return "n%d_m%d" % (int(math.log2(max(n_total, 1))), int(math.log2(max(n_total // max(n_trees, 1), 1))))


def default_cache_path():
    return os.environ.get("DAFMM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "dafmm", "autotune.json"))


class Cache:
    """A JSON file of {key: {"max_leaf": s, "leaf_warps": w, "ms": t}}; written atomically."""

    def __init__(self, path=None):
        self.path = path or default_cache_path()
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key):
        return self.data.get(key)

    def put(self, key, value):
        self.data[key] = value
        d = os.path.dirname(self.path) or "."
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune_")
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def make_key(device_name, order, precision, n_total, n_trees):
    return "%s|p%d|%s|%s" % (device_name, order, precision, size_class(n_total, n_trees))


def tune_forest(ctx, xyz, q, offsets, order, precision="fp32", cache=None, reps=2, force=False):
    """Best (max_leaf, leaf_warps) for solving the forest (xyz, q, offsets) at `order`:
    build + one evaluation, timed per candidate (device inputs recommended).  Returns
    {"max_leaf", "leaf_warps", "ms", "cached", "trials"} and leaves the winning tile set on
    the context."""
    import torch
    cache = cache if cache is not None else Cache()
    offsets = np.asarray(offsets, dtype=np.int64)
    n_total, n_trees = int(offsets[-1]), len(offsets) - 1
    key = make_key(torch.cuda.get_device_name(), order, precision, n_total, n_trees)
    hit = cache.get(key)
    if hit is not None and not force:
        B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, hit["leaf_warps"])
        return dict(hit, cached=True, trials=[])
    dev = torch.device("cuda", torch.cuda.current_device())
    phi = torch.empty(n_total, dtype=torch.float64, device=dev)
    E = torch.empty((n_total, 3), dtype=torch.float64, device=dev)
    trials = []
    best = None
    for s in leaf_candidates(order):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = ctx.build_forest(xyz, q, offsets, max_leaf=s)
        torch.cuda.synchronize()
        build_ms = (time.perf_counter() - t0) * 1e3
        for w in LEAF_WARPS:
            B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, w)
            f.eval(order, phi, E, precision=precision)  # warm (tables, expansions)
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                f.eval(order, phi, E, precision=precision)
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            total = build_ms + min(ms)
            trials.append({"max_leaf": s, "leaf_warps": w, "build_ms": build_ms, "eval_ms": min(ms)})
            if best is None or total < best["ms"]:
                best = {"max_leaf": s, "leaf_warps": w, "ms": total}
        f.free()
    B.dafmm_sync(ctx.h)
    cache.put(key, best)
    B.dafmm_set_option(ctx.h, B.DAFMM_OPT_LEAF_WARPS, best["leaf_warps"])
    return dict(best, cached=False, trials=trials)
