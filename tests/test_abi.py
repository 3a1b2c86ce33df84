"""The C-ABI library loads and exports every entry point include/dafmm.h declares (no
compute calls: these run without a GPU), and the binding covers the same names."""
import ctypes
import os
import re

import pytest

from paper_2508_02626_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "dafmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dafmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    assert set(declared_entry_points()) == set(binding.SIGNATURES)
    for n in declared_entry_points():
        assert callable(getattr(binding, n))


def test_footprint_is_monotone_and_rejects_bad_order():
    binding.load()
    a = binding.dafmm_footprint(10_000, 6, 3)
    b = binding.dafmm_footprint(1_000_000, 8, 5)
    c = binding.dafmm_footprint(1_000_000, 10, 5)
    assert 0 < a < b < c
    assert binding.dafmm_footprint(1000, 11, 3) == 0


def test_no_device_is_reported_not_crashed():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(binding.DafmmError) as e:
        binding.dafmm_create(0)
    assert e.value.code == binding.DAFMM_ERR_NO_DEVICE
