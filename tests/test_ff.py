"""Float-float arithmetic (csrc/ff.cuh) on the host: the sum, product, 1/sqrt and reciprocal of
pairs of FP32 numbers against long double over random operands of magnitudes 2^-20..2^20 and
both signs, held to the published bounds of the double-word algorithms (3 u^2 for the sum,
5 u^2 for the product, u = 2^-24) and to 1e-13 for the Newton-refined 1/sqrt and 1/x; and the
generated P2M and L2P of orders 2..10 evaluated in float-float against FP64 (within 1e-12 of
the largest coefficient, the bound the FP64 operators are held to against the oracle)."""
import os
import subprocess
import tempfile

from paper_2508_02626_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U = 2.0 ** -24


def test_float_float_arithmetic():
    gen_dir = _build.generate()
    d = tempfile.mkdtemp(prefix="dafmm_ff_")
    exe = os.path.join(d, "ffc")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-I", os.path.dirname(gen_dir),
                           "-o", exe, os.path.join(ROOT, "tests", "ff_check.cpp")])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    e = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert e["add"] <= 3 * U * U and e["cancel"] <= 3 * U * U, e
    assert e["mul"] <= 5 * U * U, e
    assert e["rsqrt"] <= 1e-13 and e["rcp"] <= 1e-13, e
    assert e["gen_p2m"] <= 1e-12 and e["gen_l2p"] <= 1e-12, e
