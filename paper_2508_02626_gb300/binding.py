"""ctypes binding of libdafmm.so (include/dafmm.h), argument marshalling only.

Every function carries the name of the C entry point it wraps.  Arrays may be torch
tensors (CPU or CUDA) or numpy arrays; the library itself tells host from device
memory.  There is no Python fallback: if the compiled library is missing, loading
raises ``RuntimeError``.
"""
import ctypes
import os

import numpy as np

from . import _build

DAFMM_OK = 0
DAFMM_ERR_INVALID_ARG = -1
DAFMM_ERR_UNSUPPORTED_ORDER = -2
DAFMM_ERR_OVER_BUDGET = -3
DAFMM_ERR_CUDA = -4
DAFMM_ERR_TIMEOUT = -5
DAFMM_ERR_UNSUPPORTED = -6
DAFMM_ERR_NO_DEVICE = -7
DAFMM_ERR_CANCELLED = -8
DAFMM_ERR_CHECK = -9

DAFMM_FP64 = 0
DAFMM_MIXED = 1
DAFMM_FP32 = 2
DAFMM_FF = 3
PRECISIONS = {"fp64": DAFMM_FP64, "mixed": DAFMM_MIXED, "fp32": DAFMM_FP32, "ff": DAFMM_FF}
DAFMM_OP_NUMERICAL_DA = 16  # or-ed into the precision of a single-operator batch
MAX_ORDER = 10

# entry points declared in include/dafmm.h: name -> (restype, argtypes)
_vp, _i, _i64, _sz, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "dafmm_create": (_i, [ctypes.POINTER(_vp), _i, _sz]),
    "dafmm_destroy": (None, [_vp]),
    "dafmm_last_error": (ctypes.c_char_p, [_vp]),
    "dafmm_bytes_in_use": (_sz, [_vp]),
    "dafmm_build_tree": (_i, [_vp, _vp, _vp, _i64, _vp, _i, _i, _vp, ctypes.POINTER(_vp)]),
    "dafmm_tree_free": (_i, [_vp]),
    "dafmm_tree_info": (_i, [_vp, _vp, _vp]),
    "dafmm_eval": (_i, [_vp, _i, _d, _i, _vp, _vp, _vp]),
    "dafmm_footprint": (_sz, [_i64, _i, _i, _i, _i]),
    "dafmm_set_profiling": (_i, [_vp, _i]),
    "dafmm_set_option": (_i, [_vp, _i, _i64]),
    "dafmm_sync": (_i, [_vp, _vp]),
    "dafmm_debug_expire_wait": (_i, [_vp, _vp]),
    "dafmm_debug_check": (_i, [_vp, _vp]),
    "dafmm_eval_noalloc": (_i, [_vp, _i, _vp, _vp, _vp]),
    "dafmm_probe_peak": (_i, [_i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "dafmm_debug_level": (_i64, [_vp, _i, _i, _vp, _i64]),
    "dafmm_last_phase_ms": (_i, [_vp, _vp]),
    "dafmm_op_p2m": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_op_p2l": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_op_l2p": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_op_m2p": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_op_m2m": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_op_l2l": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_op_m2l_matrix": (_i, [_vp, _i, _vp, _vp, _vp]),
    "dafmm_op_m2l": (_i, [_vp, _i, _i, _i64, _vp, _vp, _vp, _vp]),
    "dafmm_create_pooled": (_i, [ctypes.POINTER(_vp), _i, _sz]),
    "dafmm_build_forest": (_i, [_vp, _vp, _vp, _vp, _i, _vp, _i, _vp, ctypes.POINTER(_vp)]),
    "dafmm_forest_info": (_i, [_vp, _vp, _vp]),
    "dafmm_graph_create": (_i, [_vp, _i, _i, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "dafmm_graph_launch": (_i, [_vp, _vp]),
    "dafmm_graph_nodes": (_i, [_vp]),
    "dafmm_graph_free": (_i, [_vp]),
    "dafmm_server_create": (_i, [_i, _sz, _i, _i, _i64, ctypes.POINTER(_vp)]),
    "dafmm_server_submit": (_i, [_vp, _vp, _vp, _i64, _i, _i, _i, _vp, _vp, ctypes.POINTER(_i64)]),
    "dafmm_server_wait": (_i, [_vp, _i64, _d, _vp]),
    "dafmm_server_stats": (_i, [_vp, _vp]),
    "dafmm_server_last_error": (ctypes.c_char_p, [_vp]),
    "dafmm_server_destroy": (_i, [_vp]),
}

_lib = None


def library_path():
    return _build.LIB_PATH


def _open(path):
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(build_if_missing=False):
    """Load libdafmm.so.  Raises RuntimeError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libdafmm.so is not built (run __graft_entry__.build()); there is no fallback")
    _lib = _open(path)
    return _lib


def load_checked(build_if_missing=True):
    """The checked build, libdafmm_check.so (compiled with -DDAFMM_CHECK; built on first use)."""
    path = _build.CHECK_LIB_PATH
    if build_if_missing:
        _build.build(checked=True)
    elif not os.path.exists(path):
        raise RuntimeError("libdafmm_check.so is not built")
    return _open(path)


def swap_library(lib):
    """Route every wrapper of this module to `lib` (a library from load / load_checked, or None
    for the default); returns the one routed to before.  Handles made by one library must not
    be passed to another."""
    global _lib
    old, _lib = _lib, lib
    return old


class DafmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


def _ptr(a):
    """Address of a torch tensor / numpy array (None for None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or a numpy array")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(ctx, rc):
    if rc != DAFMM_OK:
        msg = load().dafmm_last_error(ctx).decode() if ctx else "dafmm call failed"
        raise DafmmError(rc, msg)


# ---- entry points ---------------------------------------------------------------------------
def dafmm_create(device=0, hbm_budget_bytes=0):
    h = _vp()
    rc = load().dafmm_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
    if rc != DAFMM_OK:
        raise DafmmError(rc, "dafmm_create failed")
    return h.value


def dafmm_create_pooled(device, pool_bytes):
    h = _vp()
    rc = load().dafmm_create_pooled(ctypes.byref(h), int(device), int(pool_bytes))
    if rc != DAFMM_OK:
        raise DafmmError(rc, "dafmm_create_pooled failed")
    return h.value


def dafmm_destroy(ctx):
    load().dafmm_destroy(ctx)


def dafmm_last_error(ctx):
    return load().dafmm_last_error(ctx).decode()


def dafmm_bytes_in_use(ctx):
    return load().dafmm_bytes_in_use(ctx)


def dafmm_build_tree(ctx, xyz, q, domain=None, uniform_depth=-1, max_leaf=64, stream=None):
    n = int(q.shape[0]) if q is not None else 0
    dom = None
    if domain is not None:
        dom = np.ascontiguousarray(domain, dtype=np.float64)
    h = _vp()
    rc = load().dafmm_build_tree(ctx, _ptr(xyz), _ptr(q), n, _ptr(dom), int(uniform_depth), int(max_leaf),
                                 _stream_ptr(stream), ctypes.byref(h))
    _check(ctx, rc)
    return h.value


def dafmm_tree_free(tree):
    load().dafmm_tree_free(tree)


def dafmm_build_forest(ctx, xyz, q, offsets, domains=None, max_leaf=64, stream=None):
    """offsets: ntrees + 1 particle offsets (host); domains: ntrees x 4 root cubes or None."""
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    dom = None if domains is None else np.ascontiguousarray(domains, dtype=np.float64).reshape(-1, 4)
    h = _vp()
    rc = load().dafmm_build_forest(ctx, _ptr(xyz), _ptr(q), offs.ctypes.data, len(offs) - 1, _ptr(dom),
                                   int(max_leaf), _stream_ptr(stream), ctypes.byref(h))
    _check(ctx, rc)
    return h.value


def dafmm_forest_info(tree):
    nt = ctypes.c_int(0)
    if load().dafmm_forest_info(tree, ctypes.byref(nt), None) != DAFMM_OK:
        raise DafmmError(DAFMM_ERR_INVALID_ARG, "dafmm_forest_info failed")
    dom = np.zeros((nt.value, 4))
    load().dafmm_forest_info(tree, None, dom.ctypes.data)
    return nt.value, dom


def dafmm_graph_create(ctx, tree, order, precision, phi=None, field=None, stream=None):
    h = _vp()
    rc = load().dafmm_graph_create(tree, int(order), int(precision), _ptr(phi), _ptr(field), _stream_ptr(stream),
                                   ctypes.byref(h))
    _check(ctx, rc)
    return h.value


def dafmm_graph_launch(ctx, graph, stream=None):
    _check(ctx, load().dafmm_graph_launch(graph, _stream_ptr(stream)))


def dafmm_graph_nodes(graph):
    return load().dafmm_graph_nodes(graph)


def dafmm_graph_free(graph):
    load().dafmm_graph_free(graph)


def dafmm_tree_info(tree):
    info = np.zeros(8, dtype=np.int64)
    dom = np.zeros(4)
    rc = load().dafmm_tree_info(tree, info.ctypes.data, dom.ctypes.data)
    if rc != DAFMM_OK:
        raise DafmmError(rc, "dafmm_tree_info failed")
    keys = ["n", "depth", "leaves", "boxes", "max_per_leaf", "adaptive", "m2l_pairs", "p2p_leaf_pairs"]
    out = {k: int(v) for k, v in zip(keys, info)}
    out["domain"] = dom
    return out


def dafmm_eval(ctx, tree, order, phi=None, field=None, theta=1.0, precision=DAFMM_FP64, stream=None):
    rc = load().dafmm_eval(tree, int(order), float(theta), int(precision), _ptr(phi), _ptr(field),
                           _stream_ptr(stream))
    _check(ctx, rc)


DAFMM_OPT_M2L_KERNEL = 1
DAFMM_OPT_TC_MASK = 2
DAFMM_OPT_LEAF_WARPS = 3
DAFMM_OPT_M2L_F16 = 4
DAFMM_OPT_M2L_ROTATION = 5
DAFMM_OPT_M2L_HARMONIC = 6


def dafmm_set_option(ctx, option, value):
    _check(ctx, load().dafmm_set_option(ctx, int(option), int(value)))


def dafmm_sync(ctx, stream=None):
    _check(ctx, load().dafmm_sync(ctx, _stream_ptr(stream)))


def dafmm_debug_expire_wait(ctx, stream=None):
    _check(ctx, load().dafmm_debug_expire_wait(ctx, _stream_ptr(stream)))


def dafmm_debug_check(ctx, stream=None):
    _check(ctx, load().dafmm_debug_check(ctx, _stream_ptr(stream)))


def dafmm_eval_noalloc(ctx, tree, order, phi=None, field=None, stream=None):
    """FP64 evaluation that allocates no device memory (order <= 6, depth <= 4, device outputs)."""
    _check(ctx, load().dafmm_eval_noalloc(tree, int(order), _ptr(phi), _ptr(field), _stream_ptr(stream)))


PEAK_KINDS = {"ffma": 0, "ffma2": 1, "dfma": 2, "rsqrt": 3, "mma_tf32": 4, "mma_f16": 5}


def dafmm_probe_peak(device, kind):
    """Measured unit rate of the GPU (operations per second) and the timed launch's ms."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load().dafmm_probe_peak(int(device), PEAK_KINDS[kind] if isinstance(kind, str) else int(kind),
                                 ctypes.byref(rate), ctypes.byref(ms))
    if rc != DAFMM_OK:
        raise DafmmError(rc, "dafmm_probe_peak(%s) failed" % kind)
    return rate.value, ms.value


DEBUG_ARRAYS = {"M": 0, "L": 1, "Mhi": 2, "Mlo": 3, "Lhi": 4, "Llo": 5}


def dafmm_debug_level(tree, which, level, ncp):
    """Copy of one level of an internal expansion array of the last evaluation, (8^l, ncp)."""
    out = np.zeros((8 ** level, ncp))
    rc = load().dafmm_debug_level(tree, DEBUG_ARRAYS[which], int(level), out.ctypes.data, out.size)
    if rc < 0:
        raise DafmmError(int(rc), "dafmm_debug_level failed")
    return out


def dafmm_set_profiling(ctx, enable):
    _check(ctx, load().dafmm_set_profiling(ctx, int(bool(enable))))


PHASES = ["p2m", "m2m", "m2l", "m2l_finest", "l2l", "leaf", "convert", "total", "launches"]


def dafmm_last_phase_ms(ctx):
    out = np.zeros(10)
    _check(ctx, load().dafmm_last_phase_ms(ctx, out.ctypes.data))
    return dict(zip(PHASES, out[:9].tolist()))


def dafmm_footprint(n, order, uniform_depth=-1, max_leaf=64, precision=DAFMM_FP64):
    return load().dafmm_footprint(int(n), int(order), int(uniform_depth), int(max_leaf), int(precision))


def _op(name, ctx, order, precision, count, a, b, out, stream):
    fn = getattr(load(), name)
    _check(ctx, fn(ctx, int(order), int(precision), int(count), _ptr(a), _ptr(b), _ptr(out), _stream_ptr(stream)))


def dafmm_op_p2m(ctx, order, precision, s, q, out, stream=None):
    _op("dafmm_op_p2m", ctx, order, precision, q.shape[0], s, q, out, stream)


def dafmm_op_p2l(ctx, order, precision, w, q, out, stream=None):
    _op("dafmm_op_p2l", ctx, order, precision, q.shape[0], w, q, out, stream)


def dafmm_op_l2p(ctx, order, precision, L, x, out4, stream=None):
    _op("dafmm_op_l2p", ctx, order, precision, x.shape[0], L, x, out4, stream)


def dafmm_op_m2p(ctx, order, precision, M, s, out4, stream=None):
    _op("dafmm_op_m2p", ctx, order, precision, s.shape[0], M, s, out4, stream)


def dafmm_op_m2m(ctx, order, precision, oct_, inp, out, stream=None):
    _op("dafmm_op_m2m", ctx, order, precision, oct_.shape[0], oct_, inp, out, stream)


def dafmm_op_l2l(ctx, order, precision, oct_, inp, out, stream=None):
    _op("dafmm_op_l2l", ctx, order, precision, oct_.shape[0], oct_, inp, out, stream)


def dafmm_op_m2l(ctx, order, precision, r0, M, out, stream=None):
    """M2L (Eq. 5) of each row of M for the displacement r0[i] (numerical DA only)."""
    _op("dafmm_op_m2l", ctx, order, precision, r0.shape[0], r0, M, out, stream)


def dafmm_op_m2l_matrix(ctx, order, v, K, stream=None):
    v = np.ascontiguousarray(v, dtype=np.int32)
    _check(ctx, load().dafmm_op_m2l_matrix(ctx, int(order), v.ctypes.data, _ptr(K), _stream_ptr(stream)))


# ---- a small convenience layer ----------------------------------------------------------------
class Context:
    """Owns a dafmm context; trees built from it are freed with it.  pool_bytes > 0 makes a
    pooled context (one reservation, no cudaFree while it lives)."""

    def __init__(self, device=0, hbm_budget_bytes=0, pool_bytes=0):
        self.h = dafmm_create_pooled(device, pool_bytes) if pool_bytes else dafmm_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            dafmm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def build_tree(self, xyz, q, domain=None, uniform_depth=-1, max_leaf=64, stream=None):
        return Tree(self, dafmm_build_tree(self.h, xyz, q, domain, uniform_depth, max_leaf, stream))

    def build_forest(self, xyz, q, offsets, domains=None, max_leaf=64, stream=None):
        return Tree(self, dafmm_build_forest(self.h, xyz, q, offsets, domains, max_leaf, stream))


class Tree:
    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def info(self):
        return dafmm_tree_info(self.h)

    def eval(self, order, phi=None, field=None, precision="fp64", theta=1.0, stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        dafmm_eval(self.ctx.h, self.h, order, phi, field, theta, prec, stream)

    def forest(self):
        return dafmm_forest_info(self.h)

    def graph(self, order, phi=None, field=None, precision="fp32", stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        return Graph(self.ctx, dafmm_graph_create(self.ctx.h, self.h, order, prec, phi, field, stream))

    def free(self):
        if self.h and self.ctx.h:
            dafmm_tree_free(self.h)
        self.h = None


class Graph:
    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def launch(self, stream=None):
        dafmm_graph_launch(self.ctx.h, self.h, stream)

    def nodes(self):
        return dafmm_graph_nodes(self.h)

    def free(self):
        if self.h:
            dafmm_graph_free(self.h)
        self.h = None


# ---- serving ------------------------------------------------------------------------------------
SERVER_STATS = ["completed", "failed", "queued", "running", "jobs", "requests_per_job", "peak_bytes",
                "peak_running"]


def dafmm_server_create(device=0, pool_bytes=8 << 30, slots=4, max_batch=64, max_job_particles=1 << 21):
    h = _vp()
    rc = load().dafmm_server_create(int(device), int(pool_bytes), int(slots), int(max_batch), int(max_job_particles),
                                    ctypes.byref(h))
    if rc != DAFMM_OK:
        raise DafmmError(rc, "dafmm_server_create failed")
    return h.value


def dafmm_server_submit(server, xyz, q, order, precision, max_leaf, phi, field):
    rid = ctypes.c_int64(0)
    rc = load().dafmm_server_submit(server, _ptr(xyz), _ptr(q), int(q.shape[0]), int(order), int(precision),
                                    int(max_leaf), _ptr(phi), _ptr(field), ctypes.byref(rid))
    if rc != DAFMM_OK:
        raise DafmmError(rc, "dafmm_server_submit failed")
    return rid.value


def dafmm_server_wait(server, rid, timeout=-1.0):
    """(status, [latency, queue, device] ms)."""
    t = np.zeros(3)
    st = load().dafmm_server_wait(server, int(rid), float(timeout), t.ctypes.data)
    return st, t


def dafmm_server_stats(server):
    out = np.zeros(8)
    load().dafmm_server_stats(server, out.ctypes.data)
    return dict(zip(SERVER_STATS, out.tolist()))


def dafmm_server_last_error(server):
    return load().dafmm_server_last_error(server).decode()


def dafmm_server_destroy(server):
    load().dafmm_server_destroy(server)


class Server:
    """A request loop with continuous batching (dafmm_server_*).  Inputs and outputs are kept
    in page-locked host tensors until the request has been waited for."""

    def __init__(self, device=0, pool_bytes=8 << 30, slots=4, max_batch=64, max_job_particles=1 << 21):
        import torch  # page-locked buffers
        self._torch = torch
        self.h = dafmm_server_create(device, pool_bytes, slots, max_batch, max_job_particles)
        self._live = {}

    def _pinned(self, a, shape):
        torch = self._torch
        if isinstance(a, torch.Tensor) and a.dtype == torch.float64 and (a.is_cuda or a.is_pinned()) \
                and a.is_contiguous():
            return a
        t = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        t.copy_(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).reshape(shape))
        return t

    def submit(self, xyz, q, order, precision="fp32", max_leaf=64, field=True, out=None):
        """out: optional (phi, field) page-locked float64 tensors to receive the result."""
        torch = self._torch
        n = int(q.shape[0])
        x = self._pinned(xyz, (n, 3))
        qq = self._pinned(q, (n,))
        if out is not None:
            phi, E = out
        else:
            phi = torch.empty(n, dtype=torch.float64, pin_memory=True)
            E = torch.empty((n, 3), dtype=torch.float64, pin_memory=True) if field else None
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        rid = dafmm_server_submit(self.h, x, qq, order, prec, max_leaf, phi, E)
        self._live[rid] = (x, qq, phi, E)
        return rid

    def wait(self, rid, timeout=-1.0):
        """(status, phi, field, {latency_ms, queue_ms, device_ms}); status DAFMM_ERR_TIMEOUT keeps
        the request pending."""
        st, t = dafmm_server_wait(self.h, rid, timeout)
        if st == DAFMM_ERR_TIMEOUT:
            return st, None, None, None
        live = self._live.pop(rid, None)
        if live is None:  # an id this server object does not hold
            return st, None, None, None
        _, _, phi, E = live
        times = dict(latency_ms=t[0], queue_ms=t[1], device_ms=t[2])
        return st, phi.numpy(), (E.numpy() if E is not None else None), times

    def stats(self):
        return dafmm_server_stats(self.h)

    def last_error(self):
        return dafmm_server_last_error(self.h)

    def close(self):
        if self.h:
            dafmm_server_destroy(self.h)
            self.h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
