"""Host structure of the M2L by rotation (Sec. 3.4), no GPU: the axial matrix's sparsity rule
row by row against the coefficient layout built from its definition; the kernel's per-lane
task lists (every output in exactly one lane, whole and in order, padding only after the real
tasks, lanes balanced to within one output); and the substitution steps run as the kernel
runs them, checked pointwise against the substituted polynomial on random data."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp(prefix="dafmm_rot_")
    so = os.path.join(d, "rot.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "paper_2508_02626_gb300", "csrc"),
                           "-o", so, os.path.join(ROOT, "tests", "rot_lists_check.cpp")])
    h = ctypes.CDLL(so)
    h.rot_lists_check.argtypes = [ctypes.c_int, ctypes.c_uint]
    h.rot_lists_check.restype = ctypes.c_int
    h.rot_lists_check_harm.argtypes = [ctypes.c_int, ctypes.c_uint]
    h.rot_lists_check_harm.restype = ctypes.c_int
    h.rot_real_tasks.argtypes = [ctypes.c_int]
    h.rot_real_tasks.restype = ctypes.c_long
    h.rot_real_tasks_harm.argtypes = [ctypes.c_int]
    h.rot_real_tasks_harm.restype = ctypes.c_long
    return h


@pytest.mark.parametrize("p", [0, 1, 2, 3, 5, 8, 10])
def test_rotation_structure_and_lists(lib, p):
    assert lib.rot_lists_check(p, 1000 + p) == 0



@pytest.mark.parametrize("p", [0, 1, 2, 3, 5, 8, 10])
def test_harmonic_lists(lib, p):
    """The harmonic lists: only the outputs of z exponent <= 1, each equal to the full lists'
    value; the z and axial steps read no input of z exponent >= 2."""
    assert lib.rot_lists_check_harm(p, 2000 + p) == 0


def test_harmonic_form_saves_work():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for p, bound in ((4, 0.75), (8, 0.5), (10, 0.4)):
        full, harm = bench.rotation_madds_per_pair(p, False), bench.rotation_madds_per_pair(p, True)
        assert harm < bound * full, (p, harm, full)


def test_bench_counts_match_the_lists(lib):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for p in (2, 4, 8, 10):
        assert bench.rotation_madds_per_pair(p, False) == lib.rot_real_tasks(p)
        assert bench.rotation_madds_per_pair(p, True) == lib.rot_real_tasks_harm(p)
