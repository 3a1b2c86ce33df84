"""Host-side AddressSanitizer and UndefinedBehaviorSanitizer runs (no GPU).

The oracle's C sources, the host build of the generated operator code and the host-side
runtime headers (pool arena, admission policy, rotation task lists, record layout, through
their CPU checks) are compiled with
-fsanitize=address,undefined, loaded in a child Python process with the ASan runtime
preloaded, and driven through every operator and orders 0..10.  The oracle also runs the
direct sum and FMM solves on uniform, adaptive, rotation-mode and depth-capped trees.  A run
passes when the child exits 0 and prints no sanitizer report.  A planted heap overflow and a
planted signed overflow, built the same way, must be reported, which shows that the harness
does catch errors."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-g"]


def _runtime():
    try:
        path = subprocess.check_output(["gcc", "-print-file-name=libasan.so"], text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("gcc not available")
    if not os.path.isabs(path) or not os.path.exists(path):
        pytest.skip("no ASan runtime")
    return path


def _run(script, extra_env):
    env = dict(os.environ)
    env.update({"LD_PRELOAD": _runtime(), "ASAN_OPTIONS": "detect_leaks=0",
                "UBSAN_OPTIONS": "halt_on_error=1:print_stacktrace=1"})
    env.update(extra_env)
    return subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=900)


def _clean(r):
    text = r.stdout + r.stderr
    return r.returncode == 0 and "AddressSanitizer" not in text and "runtime error" not in text


@pytest.fixture(scope="module")
def builds():
    _runtime()
    d = tempfile.mkdtemp(prefix="dafmm_san_")
    oracle_so = os.path.join(d, "liboracle_san.so")
    src = [os.path.join(ROOT, "oracle", f) for f in ("tpsa.c", "ops.c", "direct.c", "tree.c", "fmm.c")]
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-pthread", "-fno-fast-math", "-ffp-contract=off"]
                          + SAN + ["-o", oracle_so] + src + ["-lm"])
    from paper_2508_02626_gb300 import _build
    gen_dir = _build.generate()
    hc_so = os.path.join(d, "hc_san.so")
    # no debug information for the (large) generated code: it triples the compile time
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off"] + SAN[:-1]
                          + ["-g0", "-I", os.path.dirname(gen_dir), "-o", hc_so,
                             os.path.join(ROOT, "tests", "gen_host_check.cpp")])
    planted = os.path.join(d, "planted.so")
    with open(os.path.join(d, "planted.c"), "w") as f:
        f.write("#include <stdlib.h>\n"
                "int heap_overflow(int n) { int* a = malloc(4 * n); a[n] = 1; int r = a[0]; free(a); return r; }\n"
                "int signed_overflow(int x) { return x + 2147483647; }\n")
    subprocess.check_call(["gcc", "-O0", "-fPIC", "-shared"] + SAN + ["-o", planted, os.path.join(d, "planted.c")])
    # the host-side runtime pieces (pool arena, admission policy, rotation task lists, particle
    # record layout), through their CPU checks
    host = {}
    for name, extra in (("arena_check", []), ("serve_policy_check", []), ("rot_lists_check", []),
                        ("xq_layout_check", ["-x", "c++", "-I", "/usr/local/cuda/include"])):
        if name == "xq_layout_check" and not os.path.exists("/usr/local/cuda/include/vector_types.h"):
            continue
        so = os.path.join(d, name + ".so")
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared"] + SAN + extra
                              + ["-I", os.path.join(ROOT, "paper_2508_02626_gb300", "csrc"), "-o", so,
                                 os.path.join(ROOT, "tests", name + ".cpp")])
        host[name] = so
    return {"oracle": oracle_so, "hc": hc_so, "planted": planted, "host": host}


ORACLE_SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, '.')
import oracle as O
rng = np.random.default_rng(0)
for p in range(0, 11):
    s = rng.uniform(-0.5, 0.5, (12, 3)); q = rng.uniform(-1, 1, 12)
    M = O.p2m(p, s, q)
    O.m2m(p, M, [0.5, -0.5, 0.5])
    L = O.m2l(p, M, [2.0, 1.0, -3.0])
    O.m2l_rot(p, M, [2.0, 1.0, -3.0]); O.m2l_rot(p, M, [3.0, 0.0, 0.0])
    O.m2l_matrix(p, [3.0, 0.0, 2.0]); O.m2l_map(p, [2.0, -2.0, 1.0])
    O.p2l(p, s + 3.0, q); O.l2l(p, L, [0.25, 0.25, -0.25])
    O.l2p(p, L, s); O.m2p(p, M, s + 2.5)
    O.da_rinv(p, [1.0, 1.0, 1.0])
x = rng.random((3000, 3)); q = rng.uniform(-1, 1, 3000)
O.direct(x, q, targets=np.arange(100))
for depth in (0, 2, 3):
    O.fmm(x, q, [0, 0, 0, 1], 4, uniform_depth=depth)
O.fmm(x, q, [0, 0, 0, 1], 6, max_leaf=20)
O.fmm(x, q, [0, 0, 0, 1], 5, uniform_depth=3, m2l_mode=2)
O.fmm(x, q, [0, 0, 0, 1], 4, max_leaf=1, max_depth=8, targets=np.arange(50))
O.fmm(x[:1], q[:1], [0, 0, 0, 1], 4, max_leaf=8)
print("oracle ok")
"""

HC_SCRIPT = r"""
import ctypes, os, sys
import numpy as np
lib = ctypes.CDLL(os.environ["HC_LIB"])
D = ctypes.POINTER(ctypes.c_double)
def P(a):
    return a.ctypes.data_as(D)
for nm, args in {"hc_p2m": [ctypes.c_int, ctypes.c_int, D, ctypes.c_double, D, ctypes.c_int],
                 "hc_p2l": [ctypes.c_int, ctypes.c_int, D, ctypes.c_double, D, ctypes.c_int],
                 "hc_l2p": [ctypes.c_int, ctypes.c_int, D, D, D, ctypes.c_int],
                 "hc_m2p": [ctypes.c_int, ctypes.c_int, D, D, D, ctypes.c_int],
                 "hc_m2lmap": [ctypes.c_int, D, D, D],
                 "hc_shift": [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, ctypes.c_int]}.items():
    getattr(lib, nm).argtypes = args
    getattr(lib, nm).restype = ctypes.c_int
rng = np.random.default_rng(1)
for p in range(0, 11):
    nc = (p + 1) * (p + 2) * (p + 3) // 6
    for prec in (64, 32):
        s = rng.uniform(-0.5, 0.5, 3); out = np.zeros(nc)
        assert lib.hc_p2m(p, prec, P(s), 0.5, P(out), nc) == 0
        assert lib.hc_p2l(p, prec, P(s + 2.5), 0.5, P(out), nc) == 0
        C = rng.uniform(-1, 1, nc); res = np.zeros(4)
        assert lib.hc_l2p(p, prec, P(C), P(s), P(res), nc) == 0
        assert lib.hc_m2p(p, prec, P(C), P(s + 2.5), P(res), nc) == 0
    v = np.array([2.0, -1.0, 3.0]); a, b = np.zeros(nc), np.zeros(nc)
    assert lib.hc_m2lmap(p, P(v), P(a), P(b)) == 0
    for which in (0, 1):
        for c in range(8):
            inp, out = rng.uniform(-1, 1, nc), np.zeros(nc)
            assert lib.hc_shift(p, which, c, P(inp), P(out), nc) == 0
print("generated ok")
"""


def test_oracle_is_clean(builds):
    r = _run(ORACLE_SCRIPT, {"DAFMM_ORACLE_LIB": builds["oracle"]})
    assert _clean(r) and "oracle ok" in r.stdout, r.stderr[-3000:]


def test_generated_operators_are_clean(builds):
    r = _run(HC_SCRIPT, {"HC_LIB": builds["hc"]})
    assert _clean(r) and "generated ok" in r.stdout, r.stderr[-3000:]


HOST_SCRIPT = r"""
import ctypes, json, os
libs = json.loads(os.environ["HOST_LIBS"])
C = ctypes
if "arena_check" in libs:
    a = C.CDLL(libs["arena_check"]); a.arena_check.argtypes = [C.c_int, C.c_int, C.c_ulonglong]
    assert a.arena_check(64, 4000, 1) == 0 and a.arena_check(1000, 20000, 2) == 0 and a.arena_check(7, 2000, 3) == 0
if "serve_policy_check" in libs:
    s = C.CDLL(libs["serve_policy_check"]); s.policy_check.argtypes = [C.c_int, C.c_ulonglong]
    assert s.policy_check(5000, 1) == 0
if "rot_lists_check" in libs:
    r = C.CDLL(libs["rot_lists_check"]); r.rot_lists_check.argtypes = [C.c_int, C.c_uint]
    r.rot_real_tasks.argtypes = [C.c_int]; r.rot_real_tasks.restype = C.c_long
    for p in range(11):
        assert r.rot_lists_check(p, 100 + p) == 0 and r.rot_real_tasks(p) > 0
if "xq_layout_check" in libs:
    x = C.CDLL(libs["xq_layout_check"]); x.xq_layout_check.argtypes = [C.c_uint]
    x.octmajor_check.argtypes = [C.c_int]
    assert x.xq_layout_check(1) == 0 and all(x.octmajor_check(l) == 0 for l in range(5))
print("host ok")
"""


def test_host_runtime_pieces_are_clean(builds):
    import json
    r = _run(HOST_SCRIPT, {"HOST_LIBS": json.dumps(builds["host"])})
    assert _clean(r) and "host ok" in r.stdout, r.stderr[-3000:]


@pytest.mark.parametrize("fn,report", [("heap_overflow(4)", "heap-buffer-overflow"),
                                       ("signed_overflow(5)", "runtime error")])
def test_harness_reports_planted_errors(builds, fn, report):
    script = ("import ctypes, os\nlib = ctypes.CDLL(os.environ['PLANTED'])\n"
              "print(lib.%s)\n" % fn)
    r = _run(script, {"PLANTED": builds["planted"]})
    assert r.returncode != 0 and report in (r.stdout + r.stderr)
