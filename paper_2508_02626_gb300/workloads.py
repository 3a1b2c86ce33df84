"""Seeded synthetic particle sets for the Coulomb DA-FMM workloads.

This module only draws random numbers: it holds none of the method's
arithmetic and is shared by the tests, the benchmark and the oracle legs.
All draws use NumPy's PCG64 (``default_rng(seed)``), so every consumer sees
bit-identical float64 arrays.

Workloads (the paper measures on a 3-D Gaussian with unit standard deviation,
Sec. 3.5; the other shapes stand in for the uniform and clustered problems the
benchmark configurations name):
  uniform    x ~ U[0,1)^3, q ~ U[-1,1]
  clustered  32 centres ~ U[0,1)^3, sigma_k ~ U[0.02, 0.1], each point picks a
             cluster uniformly, x = c_k + sigma_k N(0, I), q = +1
  gaussian   x ~ N(0, I), q = +1
"""
import numpy as np

UNIT_CUBE = np.array([0.0, 0.0, 0.0, 1.0])


def uniform(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3))
    q = rng.uniform(-1.0, 1.0, n)
    return x, q


def clustered(n, seed, nclusters=32, sigma=(0.02, 0.1), charges="ones"):
    rng = np.random.default_rng(seed)
    c = rng.random((nclusters, 3))
    s = rng.uniform(sigma[0], sigma[1], nclusters)
    k = rng.integers(0, nclusters, n)
    x = c[k] + s[k, None] * rng.standard_normal((n, 3))
    q = np.ones(n) if charges == "ones" else rng.uniform(-1.0, 1.0, n)
    return x, q


def gaussian(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 3)), np.ones(n)


# the five benchmark configurations ------------------------------------------------
C1 = dict(name="uniform N=1e4 p=6 depth3", n=10_000, seed=1001, order=6, uniform_depth=3, max_leaf=0)
C2 = dict(name="uniform N=1e6 p=8 depth5", n=1_000_000, seed=2002, order=8, uniform_depth=5, max_leaf=0)
C3 = dict(name="clustered N=4e6 p=10 s=64", n=4_000_000, seed=3003, order=10, uniform_depth=-1, max_leaf=64)


def make(cfg):
    if cfg["uniform_depth"] >= 0:
        x, q = uniform(cfg["n"], cfg["seed"])
        return x, q, UNIT_CUBE.copy()
    x, q = clustered(cfg["n"], cfg["seed"])
    return x, q, None


def batch_sizes(count=256, seed=4000):
    """Batch workload: N_k = round(exp(U[ln 1e3, ln 1e5])), uniform or clustered by a fair coin,
    charges U[-1,1]; solve k uses seed + k."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed + k)
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        kind = "uniform" if rng.random() < 0.5 else "clustered"
        out.append((n, kind, seed + k))
    return out


def batch_member(n, kind, seed):
    if kind == "uniform":
        return uniform(n, seed)
    return clustered(n, seed, charges="uniform")


def poisson_stream(count=2000, rate=1.0, seed=5005):
    """Serving stream: exponential inter-arrival times at `rate` requests per unit time,
    N log-uniform in [1e3, 1e6], p uniform in {4, 6, 8}, uniform or clustered by a fair coin."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    n = np.round(np.exp(rng.uniform(np.log(1e3), np.log(1e6), count))).astype(np.int64)
    p = rng.choice([4, 6, 8], count)
    kind = np.where(rng.random(count) < 0.5, "uniform", "clustered")
    seeds = seed + 1 + np.arange(count)
    return [dict(t=float(t[i]), n=int(n[i]), order=int(p[i]), kind=str(kind[i]), seed=int(seeds[i]))
            for i in range(count)]
