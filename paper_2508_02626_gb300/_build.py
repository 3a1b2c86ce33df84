"""Build steps of the package: run the symbolic-DA code generator and compile the
CUDA library (libdafmm.so) for sm_103a with nvcc.

The library is built in-tree under ``paper_2508_02626_gb300/_build/`` (git-ignored).
Translation units are compiled in parallel, one ``-gencode`` (compute_103a/sm_103a).
"""
import concurrent.futures
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
GEN_DIR = os.path.join(CSRC, "generated")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libdafmm.so")
# the checked build (-DDAFMM_CHECK: device index checks that record a site code, no trap)
CHECK_BUILD_DIR = os.path.join(PKG, "_build_check")
CHECK_LIB_PATH = os.path.join(CHECK_BUILD_DIR, "libdafmm_check.so")
MAXORD = 10

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xptxas", "-O3", "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _gen_stamp():
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(PKG, "gen"))):
        if f.endswith(".py"):
            with open(os.path.join(PKG, "gen", f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def generate(force=False):
    """Run the code generator for orders 0..MAXORD (about ten seconds); skipped when the
    generated files match the generator's sources."""
    stamp = _gen_stamp()
    stamp_file = os.path.join(GEN_DIR, ".stamp")
    if not force and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return GEN_DIR
    os.makedirs(GEN_DIR, exist_ok=True)
    subprocess.check_call([sys.executable, os.path.join(PKG, "gen", "emit.py"), "--out", GEN_DIR,
                           "--orders", "0-%d" % MAXORD], stdout=subprocess.DEVNULL)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return GEN_DIR


def _sources():
    srcs = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu") or f.endswith(".cpp")]
    return srcs


def _extra_flags():
    """Extra nvcc flags from DAFMM_NVCC_FLAGS (e.g. -DDAFMM_LEAF_SEG=128 for a tuning build)."""
    return os.environ.get("DAFMM_NVCC_FLAGS", "").split()


def _deps_mtime():
    m = 0.0
    for root, _, files in os.walk(CSRC):
        for f in files:
            m = max(m, os.path.getmtime(os.path.join(root, f)))
    inc = os.path.join(os.path.dirname(PKG), "include")
    for f in os.listdir(inc):
        m = max(m, os.path.getmtime(os.path.join(inc, f)))
    return m


def build(force=False, jobs=None, verbose=False, checked=False):
    """Generate, compile every translation unit in parallel and link libdafmm.so (checked:
    libdafmm_check.so, compiled with -DDAFMM_CHECK into its own folder)."""
    generate()
    build_dir, lib_path = (CHECK_BUILD_DIR, CHECK_LIB_PATH) if checked else (BUILD_DIR, LIB_PATH)
    flags_file = os.path.join(build_dir, ".flags")
    extra = _extra_flags() + (["-DDAFMM_CHECK"] if checked else [])
    same_flags = os.path.exists(flags_file) and open(flags_file).read() == " ".join(extra)
    if not force and same_flags and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _deps_mtime():
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", CSRC, "-I", os.path.join(os.path.dirname(PKG), "include")]
    objs = []
    cmds = []
    for s in _sources():
        o = os.path.join(build_dir, os.path.basename(s) + ".o")
        objs.append(o)
        cmds.append([nvcc] + NVCC_FLAGS + extra + inc + ["-c", s, "-o", o])
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 1))

    def run(c):
        r = subprocess.run(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        return c, r.returncode, r.stdout

    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        for c, rc, out in ex.map(run, cmds):
            if verbose and out:
                print(out)
            if rc != 0:
                raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(c), out))
    tmp = lib_path + ".tmp.%d" % os.getpid()
    link = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stdout)
    os.replace(tmp, lib_path)
    with open(flags_file, "w") as f:
        f.write(" ".join(extra))
    return lib_path
