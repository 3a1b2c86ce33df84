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


def test_checked_build_exports_every_symbol():
    """The checked build (-DDAFMM_CHECK, its own folder and library) compiles, links and
    exports the same entry points."""
    lib = ctypes.CDLL(_build.build(checked=True))
    for n in declared_entry_points():
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
    # a uniform tree's estimate covers what its build holds: particles (FP64 SoA, FP32 records
    # and remainders, permutation: 68 B each), sort keys (8 B) and the staged host inputs
    # (32 B) -- at least 108 B per particle beyond the expansions and tables
    n = 1_000_000
    assert binding.dafmm_footprint(n, 8, 5) - binding.dafmm_footprint(0, 8, 5) >= 108 * n


def test_no_device_is_reported_not_crashed():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(binding.DafmmError) as e:
        binding.dafmm_create(0)
    assert e.value.code == binding.DAFMM_ERR_NO_DEVICE


C_CONSUMER = r"""
#include <stdio.h>
#include "dafmm.h"
int main(void) {
    dafmm_ctx* ctx = NULL;
    dafmm_tree* tree = NULL;
    double xyz[6] = {0.1, 0.2, 0.3, 0.7, 0.6, 0.5}, q[2] = {1.0, -1.0}, phi[2], field[6];
    int rc = dafmm_create(&ctx, 0, 0);
    if (rc == DAFMM_OK) {
        rc = dafmm_build_tree(ctx, xyz, q, 2, NULL, 1, 64, NULL, &tree);
        if (rc == DAFMM_OK) rc = dafmm_eval(tree, 4, 1.0, DAFMM_FP64, phi, field, NULL);
        if (rc == DAFMM_OK) rc = dafmm_sync(ctx, NULL);
        if (rc == DAFMM_OK) printf("phi %.12f %.12f\n", phi[0], phi[1]);
        if (tree) dafmm_tree_free(tree);
        dafmm_destroy(ctx);
    }
    printf("rc %d null %d\n", rc, dafmm_eval(NULL, 4, 1.0, DAFMM_FP64, phi, field, NULL));
    return 0;
}
"""


def test_header_is_c99_and_a_c_program_links_and_runs(tmp_path, lib):
    """The header compiles as strict C99 and a C program linked against the library runs: on a
    machine without a GPU every call answers with an error code (no device), never a crash; with
    one, two charges give the plain Coulomb potential."""
    import subprocess
    import torch
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(_build.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-ldafmm", "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    last = out.stdout.strip().splitlines()[-1].split()
    assert last[0] == "rc" and int(last[3]) == binding.DAFMM_ERR_INVALID_ARG
    if torch.cuda.is_available():
        assert int(last[1]) == binding.DAFMM_OK
        r = ((0.1 - 0.7) ** 2 + (0.2 - 0.6) ** 2 + (0.3 - 0.5) ** 2) ** 0.5
        phi = [float(v) for v in out.stdout.split("phi")[1].split()[:2]]
        assert abs(phi[0] - (-1.0 / r)) < 1e-12 and abs(phi[1] - (1.0 / r)) < 1e-12
    else:
        assert int(last[1]) == binding.DAFMM_ERR_NO_DEVICE
