"""ctypes wrapper around the oracle library (``oracle/*.c``).

TEST INFRASTRUCTURE ONLY.  Every function takes and returns numpy float64
arrays; the arithmetic all happens in the C library, which follows the
paper's equations in plain double precision (see ``oracle/oracle.h``).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["tpsa.c", "ops.c", "direct.c", "tree.c", "fmm.c"]
_lib = None


def build(force=False):
    """Compile the oracle (gcc, plain C, -O2, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdrs = [os.path.join(_HERE, h) for h in ("oracle.h", "oracle_internal.h", "tree_internal.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs + hdrs):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        # DAFMM_ORACLE_LIB: an instrumented build of the same sources (the sanitizer tests)
        path = os.environ.get("DAFMM_ORACLE_LIB")
        if not path:
            path = build()
        _lib = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.POINTER(ctypes.c_int64)
        I32 = ctypes.POINTER(ctypes.c_int)
        c_int, c_i64, c_dbl, c_vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        sig = {
            "or_ncoef": (c_int, [c_int]),
            "or_exponents": (c_int, [c_int, c_int, I32]),
            "or_da_mul": (c_int, [c_int, D, D, D]),
            "or_da_pow": (c_int, [c_int, D, c_dbl, D]),
            "or_da_deriv": (c_int, [c_int, D, c_int, D]),
            "or_da_compose": (c_int, [c_int, D, c_int, D, D]),
            "or_da_eval": (c_dbl, [c_int, D, D]),
            "or_da_rinv": (c_int, [c_int, D, D]),
            "or_p2m": (c_int, [c_int, c_i64, D, D, D]),
            "or_m2m": (c_int, [c_int, D, D, D]),
            "or_m2l": (c_int, [c_int, D, D, D]),
            "or_m2l_matrix": (c_int, [c_int, D, D]),
            "or_m2l_rot": (c_int, [c_int, D, D, D]),
            "or_rotation": (c_int, [D, D]),
            "or_da_linmap": (c_int, [c_int, D, D, D]),
            "or_m2l_map": (c_int, [c_int, D, D, D]),
            "or_p2l": (c_int, [c_int, c_i64, D, D, D]),
            "or_l2l": (c_int, [c_int, D, D, D]),
            "or_l2p": (c_int, [c_int, D, c_i64, D, D, D]),
            "or_m2p": (c_int, [c_int, D, c_i64, D, D, D]),
            "or_direct": (c_int, [c_i64, D, D, c_i64, I64, D, D, c_int]),
            "or_tree_build": (c_vp, [c_i64, D, D, c_int, c_int, c_int]),
            "or_tree_free": (None, [c_vp]),
            "or_tree_nbox": (c_int, [c_vp]),
            "or_tree_box": (c_int, [c_vp, c_int, I64]),
            "or_tree_perm": (c_int, [c_vp, I64]),
            "or_tree_list": (c_int, [c_vp, c_int, c_int, I32, c_int]),
            "or_fmm": (c_int, [c_i64, D, D, D, c_int, c_int, c_int, c_int, c_int, c_i64, I64, D, D,
                               c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def default_threads():
    return max(1, os.cpu_count() or 1)


# ---- numerical DA ---------------------------------------------------------------
def ncoef(order):
    return _load().or_ncoef(order)


def exponents(order):
    """(ncoef, 3) int array: exponents of each coefficient in the oracle's layout."""
    lib = _load()
    nc = lib.or_ncoef(order)
    out = np.zeros((nc, 3), dtype=np.int32)
    buf = (ctypes.c_int * 3)()
    for i in range(nc):
        lib.or_exponents(order, i, buf)
        out[i] = list(buf)
    return out


def da_mul(order, a, b):
    a, b = _f64(a), _f64(b)
    c = np.zeros_like(a)
    _check(_load().or_da_mul(order, _d(a), _d(b), _d(c)), "da_mul")
    return c


def da_pow(order, a, s):
    a = _f64(a)
    c = np.zeros_like(a)
    _check(_load().or_da_pow(order, _d(a), float(s), _d(c)), "da_pow")
    return c


def da_deriv(order, a, v):
    a = _f64(a)
    c = np.zeros_like(a)
    _check(_load().or_da_deriv(order, _d(a), int(v), _d(c)), "da_deriv")
    return c


def da_compose(fo, f, go, g):
    f, g = _f64(f), _f64(g)
    out = np.zeros(ncoef(go))
    _check(_load().or_da_compose(fo, _d(f), go, _d(g), _d(out)), "da_compose")
    return out


def da_eval(order, a, x):
    a, x = _f64(a), _f64(x)
    return _load().or_da_eval(order, _d(a), _d(x))


def da_rinv(order, x0):
    x0 = _f64(x0)
    out = np.zeros(ncoef(order))
    _check(_load().or_da_rinv(order, _d(x0), _d(out)), "da_rinv")
    return out


# ---- operators --------------------------------------------------------------------
def p2m(order, s, q):
    s, q = _f64(s, (-1, 3)), _f64(q)
    M = np.zeros(ncoef(order))
    _check(_load().or_p2m(order, len(q), _d(s), _d(q), _d(M)), "p2m")
    return M


def m2m(order, M, r0):
    M, r0 = _f64(M), _f64(r0)
    out = np.zeros_like(M)
    _check(_load().or_m2m(order, _d(M), _d(r0), _d(out)), "m2m")
    return out


def m2l(order, M, r0):
    M, r0 = _f64(M), _f64(r0)
    out = np.zeros_like(M)
    _check(_load().or_m2l(order, _d(M), _d(r0), _d(out)), "m2l")
    return out


def m2l_rot(order, M, r0):
    """M2L by the rotation of Sec. 3.4 (equal to m2l up to rounding)."""
    M, r0 = _f64(M), _f64(r0)
    out = np.zeros_like(M)
    _check(_load().or_m2l_rot(order, _d(M), _d(r0), _d(out)), "m2l_rot")
    return out


def rotation(r0):
    """Q (3x3) of Sec. 3.4 with Q r0 = (|r0|, 0, 0)."""
    r0 = _f64(r0)
    Q = np.zeros(9)
    _check(_load().or_rotation(_d(r0), _d(Q)), "rotation")
    return Q.reshape(3, 3)


def da_linmap(order, a, A):
    """a composed with the linear map u -> A u."""
    a, A = _f64(a), _f64(A, (3, 3))
    out = np.zeros_like(a)
    _check(_load().or_da_linmap(order, _d(a), _d(np.ascontiguousarray(A)), _d(out)), "da_linmap")
    return out


def m2l_map(order, r0):
    """(sqrt(R), M2 as a (3, ncoef) array) of Eq. 5."""
    r0 = _f64(r0)
    nc = ncoef(order)
    sR, mp = np.zeros(nc), np.zeros(3 * nc)
    _check(_load().or_m2l_map(order, _d(r0), _d(sR), _d(mp)), "m2l_map")
    return sR, mp.reshape(3, nc)


def m2l_matrix(order, r0):
    r0 = _f64(r0)
    nc = ncoef(order)
    K = np.zeros((nc, nc))
    _check(_load().or_m2l_matrix(order, _d(r0), _d(K)), "m2l_matrix")
    return K


def p2l(order, w, q):
    w, q = _f64(w, (-1, 3)), _f64(q)
    L = np.zeros(ncoef(order))
    _check(_load().or_p2l(order, len(q), _d(w), _d(q), _d(L)), "p2l")
    return L


def l2l(order, L, r0):
    L, r0 = _f64(L), _f64(r0)
    out = np.zeros_like(L)
    _check(_load().or_l2l(order, _d(L), _d(r0), _d(out)), "l2l")
    return out


def l2p(order, L, x):
    L, x = _f64(L), _f64(x, (-1, 3))
    n = x.shape[0]
    phi, field = np.zeros(n), np.zeros((n, 3))
    _check(_load().or_l2p(order, _d(L), n, _d(x), _d(phi), _d(field)), "l2p")
    return phi, field


def m2p(order, M, s):
    M, s = _f64(M), _f64(s, (-1, 3))
    n = s.shape[0]
    phi, field = np.zeros(n), np.zeros((n, 3))
    _check(_load().or_m2p(order, _d(M), n, _d(s), _d(phi), _d(field)), "m2p")
    return phi, field


# ---- direct sum -------------------------------------------------------------------
def direct(xyz, q, targets=None, nthreads=None):
    """Eq. 1 with compensated sums.  Returns (phi, field) for the targets."""
    xyz, q = _f64(xyz, (-1, 3)), _f64(q)
    n = len(q)
    nt = n if targets is None else len(targets)
    tg = None
    if targets is not None:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
    phi, field = np.zeros(nt), np.zeros((nt, 3))
    rc = _load().or_direct(n, _d(xyz), _d(q), nt,
                           tg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if tg is not None else None,
                           _d(phi), _d(field), nthreads or default_threads())
    _check(rc, "direct")
    return phi, field


# ---- tree ---------------------------------------------------------------------------
class Tree:
    """The oracle's octree with its U/V/W/X lists (read-only view)."""

    LISTS = {"U": 0, "V": 1, "W": 2, "X": 3, "C": 4}

    def __init__(self, xyz, domain, uniform_depth=-1, max_leaf=64, max_depth=21):
        self._lib = _load()
        xyz = _f64(xyz, (-1, 3))
        dom = _f64(domain)
        self.n = xyz.shape[0]
        self._h = self._lib.or_tree_build(self.n, _d(xyz), _d(dom), int(uniform_depth), int(max_leaf),
                                          int(max_depth))
        if not self._h:
            raise ValueError("oracle tree build rejected its arguments")
        nb = self._lib.or_tree_nbox(self._h)
        info = np.zeros((nb, 8), dtype=np.int64)
        for b in range(nb):
            self._lib.or_tree_box(self._h, b, info[b].ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        self.level = info[:, 0]
        self.ijk = info[:, 1:4]
        self.parent = info[:, 4]
        self.is_leaf = info[:, 5].astype(bool)
        self.pbeg = info[:, 6]
        self.pend = info[:, 7]
        self.perm = np.zeros(self.n, dtype=np.int64)
        self._lib.or_tree_perm(self._h, self.perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))

    @property
    def nbox(self):
        return len(self.level)

    def list(self, b, which):
        k = self.LISTS[which]
        cnt = self._lib.or_tree_list(self._h, int(b), k, None, 0)
        buf = (ctypes.c_int * max(cnt, 1))()
        self._lib.or_tree_list(self._h, int(b), k, buf, cnt)
        return np.array(buf[:cnt], dtype=np.int64)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_tree_free(self._h)
            self._h = None


# ---- FMM ----------------------------------------------------------------------------
def fmm(xyz, q, domain, order, uniform_depth=-1, max_leaf=64, max_depth=21, m2l_mode=1,
        targets=None, nthreads=None):
    """The FMM traversal of Sec. 1.  Returns (phi, field) for the targets (all by default)."""
    xyz, q, dom = _f64(xyz, (-1, 3)), _f64(q), _f64(domain)
    n = len(q)
    nt = n if targets is None else len(targets)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    phi, field = np.zeros(nt), np.zeros((nt, 3))
    rc = _load().or_fmm(n, _d(xyz), _d(q), _d(dom), int(uniform_depth), int(max_leaf), int(max_depth),
                        int(order), int(m2l_mode), nt,
                        tg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if tg is not None else None,
                        _d(phi), _d(field), nthreads or default_threads())
    _check(rc, "fmm")
    return phi, field


def bounding_cube(xyz):
    """Smallest axis-aligned cube holding every point, enlarged by 1e-12 of its size on the
    upper side so that the largest coordinate falls strictly inside (domain reading of the
    design notes).  Returns [x0, y0, z0, size]."""
    xyz = _f64(xyz, (-1, 3))
    lo = xyz.min(axis=0)
    hi = xyz.max(axis=0)
    size = float((hi - lo).max())
    if size <= 0.0:
        size = 1.0
    size = size * (1.0 + 1e-12)
    return np.array([lo[0], lo[1], lo[2], size])
