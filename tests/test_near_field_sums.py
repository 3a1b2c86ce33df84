"""The summation of the FP32 near field, emulated on the CPU (numpy FP32 scalars; no code shared
with the kernels).

Each lane adds its pair terms in FP32, two sources per packed instruction, so two running
halves per group of at most 128 sources (one group per 128-record list segment).  The group's sum is folded into a compensated
(hi, lo) pair by an error-free two-sum.  Against the exact (FP64) sum of the same FP32 terms,
the result's error stays within a few FP32 units of sum |term|, whatever the list length:
27 neighbour leaves of ~30 particles, 27 leaves of 512, or 1e5 sources.  A plain FP32
running sum of 1e5 terms is an order of magnitude worse."""
import numpy as np
import pytest

U = 2.0 ** -24  # FP32 unit roundoff
F = np.float32


def terms(n, seed, signed):
    """q_j / r_j for n sources around a target, rounded to FP32 as the kernel's terms are."""
    rng = np.random.default_rng(seed)
    d = (rng.uniform(-0.5, 0.5, 3)[None, :] - rng.uniform(-1.5, 1.5, (n, 3))).astype(np.float32)
    r = np.sqrt((d.astype(np.float64) ** 2).sum(1))
    q = rng.uniform(-1.0, 1.0, n) if signed else np.ones(n)
    return (q / r).astype(np.float32)


def two_sum_add(hi, lo, v):
    s = F(hi + v)
    bp = F(s - hi)
    lo = F(lo + F(F(hi - F(s - bp)) + F(v - bp)))
    return s, lo


def near_field_sum(v, group=128):
    hi = lo = F(0)
    for g0 in range(0, len(v), group):
        a = b = F(0)  # the two halves of the packed sums
        for j, x in enumerate(v[g0:g0 + group]):
            if j % 2 == 0:
                a = F(a + x)
            else:
                b = F(b + x)
        hi, lo = two_sum_add(hi, lo, F(a + b))
    return float(hi) + float(lo)


def running_sum(v):
    s = F(0)
    for x in v:
        s = F(s + x)
    return float(s)


@pytest.mark.parametrize("n", [824, 13_824, 100_000])
@pytest.mark.parametrize("signed", [False, True])
def test_compensated_groups_keep_fp32_level(n, signed):
    v = terms(n, 11 + n, signed)
    exact = float(np.sum(v.astype(np.float64)))
    scale = float(np.sum(np.abs(v.astype(np.float64))))
    err = abs(near_field_sum(v) - exact)
    assert err <= 8 * U * scale, (err / scale)
    if not signed and n >= 13_824:
        assert abs(running_sum(v) - exact) >= 10 * err


def test_two_sum_is_error_free():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        hi, v = F(rng.normal() * 1e3), F(rng.normal())
        s, lo = two_sum_add(hi, F(0), v)
        assert float(s) + float(lo) == float(hi) + float(v)  # exact in FP64
