"""The CPU leg of bench.py that times the oracle, on the small uniform workload (N = 1e4,
depth 3, p = 6): it runs one full oracle solve without extrapolation, compares the given
results with the oracle over every particle, and with the direct sum on 2000 particles.  The
oracle's own result stands in for the GPU's here, so its error against the oracle is zero
and its error against the direct sum is the method's."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402
from paper_2508_02626_gb300 import workloads as W  # noqa: E402


def test_cpu_baseline_full_solve_small():
    cfg = W.C1
    x, q, dom = W.make(cfg)
    phi, E = O.fmm(x, q, dom, cfg["order"], uniform_depth=cfg["uniform_depth"])
    cpu, acc = bench.cpu_baseline(x, q, dom, cfg, phi, E, {cfg["order"]: phi})
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    assert "nothing extrapolated" in cpu["sample"]
    assert acc["targets"] == cfg["n"] and acc["direct_sum_targets"] == 2000
    assert acc["rel_l2_phi_vs_oracle"] == 0.0 and acc["rel_l2_field_vs_oracle"] == 0.0
    assert acc["rel_l2_phi_vs_direct"] == acc["oracle_rel_l2_phi_vs_direct"]
    # the method's own error at p = 6 on this workload: well above rounding, well below 1
    assert 1e-7 < acc["oracle_rel_l2_phi_vs_direct"] < 1e-2
    assert acc["fp64_rel_l2_phi_vs_direct_by_order"]["p6"] == acc["oracle_rel_l2_phi_vs_direct"]
    assert acc["smallest_order_reaching_1e-7"] is None
