"""The pair-interleaved FP32 particle records of the near field (tree_common.cuh), no GPU:
every leaf starts on an even record, its records and the zero record that completes an odd
leaf stay inside xq_records(n, leaves) and never overlap another leaf's, no record pair spans
two leaves (so a leaf's pairs do not depend on what precedes it in the sorted order), and
records are stored as (x, x', y, y') (z, z', q, q') and read back unchanged.  A build with a
planted mistake (leaves placed without the rounding to an even record) must fail.  The
octant-major box index of the same header is a bijection inverted by its decoder, with the 8
children of a parent at one offset of the 8 octant slabs."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


def _build(extra):
    if not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("CUDA headers not installed")
    d = tempfile.mkdtemp(prefix="dafmm_xq_")
    so = os.path.join(d, "xq.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-x", "c++",
                           "-I", os.path.join(ROOT, "paper_2508_02626_gb300", "csrc"), "-I", CUDA_INC]
                          + extra + ["-o", so, os.path.join(ROOT, "tests", "xq_layout_check.cpp")])
    h = ctypes.CDLL(so)
    h.xq_layout_check.argtypes = [ctypes.c_uint]
    h.xq_layout_check.restype = ctypes.c_int
    h.octmajor_check.argtypes = [ctypes.c_int]
    h.octmajor_check.restype = ctypes.c_int
    return h


@pytest.fixture(scope="module")
def lib():
    return _build([])


def test_record_layout(lib):
    for seed in (1, 2, 3):
        assert lib.xq_layout_check(seed) == 0


@pytest.mark.parametrize("level", [0, 1, 2, 3, 5])
def test_octant_major_index(lib, level):
    assert lib.octmajor_check(level) == 0


def test_planted_odd_base_fails():
    lib = _build(["-DPLANT_ODD_BASE"])
    assert lib.xq_layout_check(1) != 0
