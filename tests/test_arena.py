"""The pooled context's device arena (host logic, no GPU): its first-fit suballocator against
a brute-force model of 256-byte units -- same block chosen, no overlap, free neighbours
merged, accounting exact."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp(prefix="dafmm_arena_")
    so = os.path.join(d, "arena.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "paper_2508_02626_gb300", "csrc"),
                           "-o", so, os.path.join(ROOT, "tests", "arena_check.cpp")])
    h = ctypes.CDLL(so)
    h.arena_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong]
    h.arena_check.restype = ctypes.c_int
    return h


@pytest.mark.parametrize("units,steps,seed", [(64, 4000, 1), (1000, 20000, 2), (7, 2000, 3)])
def test_arena_matches_model(lib, units, steps, seed):
    assert lib.arena_check(units, steps, seed) == 0
