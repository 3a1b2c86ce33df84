"""The arithmetic of the FP32 mode's tensor-core M2L, emulated on the CPU (numpy; no code
shared with the kernels), against the FP64 contraction with the oracle's M2L matrices (Eq. 5)
and P2M multipoles (Eq. 2).

The scheme: matrix rows are scaled by a power of two shared by all displacements, each
matrix by one more, and each source multipole row by the power of two that puts its largest
magnitude in [0.5, 1).  Every operand is split into F16 parts, hi = f16(x) and
lo = f16(x - hi).  Each displacement's term is A_hi B_hi + A_hi B_lo + A_lo B_hi; the products
are exact in FP32 and are accumulated in FP32.  The term is then rescaled and added in FP32,
and the row scale is removed at the end.

The MIXED mode's TF32 splits (hi = tf32(x), lo = tf32(x - hi), no scales) are emulated the
same way.

Checked, on the potential the local expansion gives at points of the target box:
  * the error stays at the FP32 level: within 4x of a plain FP32 product of the same FP32
    multipoles, and below the FP32 mode's 3.8e-6 parity bound;
  * power-of-two scaling makes the scheme exactly invariant to the scale of the charges.
    Charges times 2^-30 or 2^20 give the same relative error, because the F16 operands are
    bit-identical.  The same split without the scales loses everything to F16 underflow, or
    overflows."""
import itertools
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

DISPLACEMENTS = [v for v in itertools.product(range(-3, 4), repeat=3) if max(map(abs, v)) >= 2]  # 316
_K = {}


def matrices(p):
    if p not in _K:
        _K[p] = np.array([O.m2l_matrix(p, np.array(v, float)) for v in DISPLACEMENTS])
    return _K[p]


def pow2_scale(m):
    """2^-e with m 2^-e in [0.5, 1) (1 for m = 0)."""
    return np.ldexp(1.0, -np.frexp(m)[1]) if m > 0 else 1.0


def split16(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float64)).astype(np.float16)
    return hi.astype(np.float32), lo.astype(np.float32)


def f16x3_local(Ks, Ms, scaled=True, products=("hh", "hl", "lh")):
    """The local expansion sum_v K_v M_v by the F16 split scheme (FP32 result as float64);
    `products` picks the split products kept (K part, M part: h = hi, l = lo)."""
    r = np.array([pow2_scale(m) for m in np.abs(Ks).max(axis=(0, 2))]) if scaled else np.ones(Ks.shape[1])
    L = np.zeros(Ks.shape[1], np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        for K, M in zip(Ks, Ms):
            Kr = K * r[:, None]
            s = pow2_scale(np.abs(Kr).max()) if scaled else 1.0
            g = pow2_scale(np.abs(M).max()) if scaled else 1.0
            Khi, Klo = split16(Kr * s)
            Mhi, Mlo = split16(M * g)
            parts = {"hh": (Khi, Mhi), "hl": (Khi, Mlo), "lh": (Klo, Mhi)}
            t = np.zeros_like(L)
            for k in products:
                t = t + parts[k][0] @ parts[k][1]
            L = L + t * np.float32(1.0 / (g * s))
        return L.astype(np.float64) / r


def workload(p, seed, charge_scale=1.0):
    """One target box with a source box of 30 random charges at each of the 316 displacements;
    multipoles stored as FP32 rows, as in the FP32 mode."""
    rng = np.random.default_rng(seed)
    Ms = np.array([O.p2m(p, rng.uniform(-0.5, 0.5, (30, 3)), charge_scale * rng.uniform(-1, 1, 30))
                   for _ in DISPLACEMENTS])
    X = rng.uniform(-0.5, 0.5, (200, 3))
    return Ms.astype(np.float32).astype(np.float64), X


def potential_error(p, L, L64, X):
    ref = O.l2p(p, L64, X)[0]
    return float(np.linalg.norm(O.l2p(p, L, X)[0] - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("p", [4, 8, 10])
@pytest.mark.parametrize("seed", [0, 1])
def test_f16_split_is_fp32_level(p, seed):
    Ks = matrices(p)
    Ms, X = workload(p, seed)
    L64 = np.einsum("vba,va->b", Ks, Ms)
    plain = np.zeros(Ks.shape[1], np.float32)
    for K, M in zip(Ks, Ms):
        plain = plain + K.astype(np.float32) @ M.astype(np.float32)
    e16 = potential_error(p, f16x3_local(Ks, Ms), L64, X)
    e32 = potential_error(p, plain.astype(np.float64), L64, X)
    assert e16 <= max(4.0 * e32, 1e-6), (e16, e32)
    assert e16 <= 3.8e-6


def tf32(x):
    """Round FP32 values to TF32 (10 mantissa bits), to nearest with ties away from zero."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def tf32x3_local(Ks, Ms):
    """The MIXED mode's M2L: operands rounded to FP32, split as hi = tf32(x), lo = tf32(x - hi)
    (TF32 keeps FP32's exponent range, so no scales), three exact products per displacement
    accumulated in FP32 and summed in FP32."""
    L = np.zeros(Ks.shape[1], np.float32)
    for K, M in zip(Ks, Ms):
        K32, M32 = K.astype(np.float32), M.astype(np.float32)
        Khi, Mhi = tf32(K32), tf32(M32)
        Klo, Mlo = tf32(K32 - Khi), tf32(M32 - Mhi)
        L = L + ((Khi @ Mhi + Khi @ Mlo) + Klo @ Mhi)
    return L.astype(np.float64)


def test_tf32_rounding():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -10)  # TF32 spacing at 1
    x = np.array([one + ulp / 4, one + ulp / 2, one + 3 * ulp / 4, -(one + ulp / 2)], np.float32)
    assert tf32(x).tolist() == [1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, -(1.0 + 2.0 ** -10)]


@pytest.mark.parametrize("p", [4, 8, 10])
def test_tf32_split_is_fp32_level(p):
    Ks = matrices(p)
    rng = np.random.default_rng(7)
    Ms = np.array([O.p2m(p, rng.uniform(-0.5, 0.5, (30, 3)), rng.uniform(-1, 1, 30)) for _ in DISPLACEMENTS])
    X = rng.uniform(-0.5, 0.5, (200, 3))
    L64 = np.einsum("vba,va->b", Ks, Ms)
    plain = np.zeros(Ks.shape[1], np.float32)
    for K, M in zip(Ks, Ms):
        plain = plain + K.astype(np.float32) @ M.astype(np.float32)
    e_tf = potential_error(p, tf32x3_local(Ks, Ms), L64, X)
    e32 = potential_error(p, plain.astype(np.float64), L64, X)
    assert e_tf <= max(4.0 * e32, 1e-6), (e_tf, e32)
    assert e_tf <= 3.8e-6


@pytest.mark.parametrize("p", [4, 8])
def test_power_of_two_scaling_is_charge_scale_invariant(p):
    Ks = matrices(p)
    errs, unscaled = [], []
    for cs in (1.0, 2.0 ** -30, 2.0 ** 20):
        Ms, X = workload(p, 3, charge_scale=cs)
        L64 = np.einsum("vba,va->b", Ks, Ms)
        errs.append(potential_error(p, f16x3_local(Ks, Ms), L64, X))
        with np.errstate(over="ignore", invalid="ignore"):
            u = potential_error(p, f16x3_local(Ks, Ms, scaled=False), L64, X)
        unscaled.append(u)
    # scaling every charge by 2^k changes the box factors only: identical F16 operands
    assert errs[1] == pytest.approx(errs[0], rel=1e-9) and errs[2] == pytest.approx(errs[0], rel=1e-9)
    # without the scales: charges at 2^-30 underflow in F16, charges at 2^20 overflow it
    assert unscaled[1] > 0.5
    assert not np.isfinite(unscaled[2]) or unscaled[2] > 0.5


@pytest.mark.parametrize("p", [4, 8, 10])
def test_two_products_miss_the_fp32_bound(p):
    """Dropping either cross product (two MMAs per term instead of three) leaves the F16
    rounding of the dropped part, about 2^-11 relative: 1e-4..1e-3 here, far above the FP32
    mode's 3.8e-6 bound, so the kernel keeps three products."""
    Ks = matrices(p)
    Ms, X = workload(p, 0)
    L64 = np.einsum("vba,va->b", Ks, Ms)
    e3 = potential_error(p, f16x3_local(Ks, Ms), L64, X)
    for keep in (("hh", "hl"), ("hh", "lh")):
        e2 = potential_error(p, f16x3_local(Ks, Ms, products=keep), L64, X)
        assert e2 > 10 * 3.8e-6 and e2 > 100 * e3, (keep, e2, e3)


@pytest.mark.parametrize("p", [4, 8, 10])
def test_harmonic_f16_split_is_fp32_level(p):
    """The same scheme in the harmonic basis (the FP32 mode's default): the matrices restricted
    to the free coefficients and composed with the expansion X, the multipoles' free
    coefficients only, the result expanded by X -- within the same bounds."""
    from test_harmonic_basis import basis
    _, free, X = basis(p)
    Ks = matrices(p)
    Kh = np.array([K[free] @ X for K in Ks])
    for seed in (0, 1):
        Ms, Xp = workload(p, seed)
        L64 = np.einsum("vba,va->b", Ks, Ms)
        plain = np.zeros(Ks.shape[1], np.float32)
        for K, M in zip(Ks, Ms):
            plain = plain + K.astype(np.float32) @ M.astype(np.float32)
        eh = potential_error(p, X @ f16x3_local(Kh, Ms[:, free]), L64, Xp)
        e32 = potential_error(p, plain.astype(np.float64), L64, Xp)
        assert eh <= max(4.0 * e32, 1e-6), (eh, e32)
        assert eh <= 3.8e-6
