"""Work counts behind bench.py's roofline figures, no GPU: the near-field interaction count
against brute force over particle pairs on a small tree, the M2L by rotation's multiply-adds
against the real tasks of the kernel's own step lists (rot_lists.h), and the near-field
roofline's arithmetic and its failure mode (an error entry, never an exception)."""
import ctypes
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_near_field_interactions_brute_force():
    rng = np.random.default_rng(5)
    x = rng.random((600, 3))
    x[:7] = [[0.0, 0.0, 0.0], [0.999999, 0.5, 0.5], [0.25, 0.25, 0.25], [0.5, 0.5, 0.5],
             [0.75, 0.0, 0.999], [0.125, 0.375, 0.625], [0.0, 1.0 - 1e-12, 0.3]]
    dom = np.array([0.0, 0.0, 0.0, 1.0])
    for depth in (0, 1, 2, 3):
        k = np.clip(np.floor(x * (1 << depth)).astype(np.int64), 0, (1 << depth) - 1)
        near = np.abs(k[:, None, :] - k[None, :, :]).max(axis=2) <= 1
        want = int(near.sum()) - len(x)  # ordered pairs i != j in adjacent or equal leaves
        assert bench.near_field_interactions(x, dom, depth) == want


def test_near_field_interactions_headline_tree():
    from paper_2508_02626_gb300 import workloads as W
    x, q, dom = W.make(W.C2)
    # N = 1e6 uniform, depth 5: about 7.74e8 interactions (32,768 leaves of ~30.5 particles)
    assert bench.near_field_interactions(x, dom, 5) == 773_378_370


@pytest.fixture(scope="module")
def rot():
    d = tempfile.mkdtemp(prefix="dafmm_rotc_")
    so = os.path.join(d, "rot.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "paper_2508_02626_gb300", "csrc"),
                           "-o", so, os.path.join(ROOT, "tests", "rot_lists_check.cpp")])
    h = ctypes.CDLL(so)
    h.rot_real_tasks.argtypes = [ctypes.c_int]
    h.rot_real_tasks.restype = ctypes.c_long
    h.rot_real_tasks_harm.argtypes = [ctypes.c_int]
    h.rot_real_tasks_harm.restype = ctypes.c_long
    return h


@pytest.mark.parametrize("p", [2, 4, 6, 8, 10])
def test_rotation_madds_match_the_kernel_lists(rot, p):
    assert bench.rotation_madds_per_pair(p, harm=False) == rot.rot_real_tasks(p)
    assert bench.rotation_madds_per_pair(p) == rot.rot_real_tasks_harm(p)


def test_near_field_roofline_arithmetic():
    x = np.random.default_rng(1).random((2000, 3))
    dom = np.array([0.0, 0.0, 0.0, 1.0])
    r = bench.near_field_roofline(x, dom, 2, 5e-4, 2000.0)  # 0.5 us: large enough to read after rounding
    inter = bench.near_field_interactions(x, dom, 2)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12, rel=1e-3)
    assert r["achieved"] == pytest.approx(18.0 * inter / 0.5e-6 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    bad = bench.near_field_roofline(np.zeros((3, 2)), dom, 2, 0.5, 2000.0)
    assert set(bad) == {"error"}
