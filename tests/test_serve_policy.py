"""The serving loop's admission policy (host logic, no GPU) on random queues: the oldest
request decides the class and is always admitted when it fits; same-class requests follow in
order up to the batch, particle and memory limits without overtaking each other; nothing is
admitted while the oldest request does not fit."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp(prefix="dafmm_policy_")
    so = os.path.join(d, "policy.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "paper_2508_02626_gb300", "csrc"),
                           "-o", so, os.path.join(ROOT, "tests", "serve_policy_check.cpp")])
    h = ctypes.CDLL(so)
    h.policy_check.argtypes = [ctypes.c_int, ctypes.c_ulonglong]
    h.policy_check.restype = ctypes.c_int
    return h


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_policy_rules(lib, seed):
    assert lib.policy_check(20000, seed) == 0
