"""ctypes binding of the C ABI in ``include/bc_gb300.h`` (argument marshalling
only: every step of the computation runs in the CUDA library).

Loading fails loudly when the library is missing or no CUDA device is
visible; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

BC_OK = 0
BC_WARN_SIGMA_OVERFLOW = 1
BC_ERR_ARG = -1
BC_ERR_NOT_SYMMETRIC = -2
BC_ERR_WEIGHT = -3
BC_ERR_OOM = -4
BC_ERR_CUDA = -5
BC_ERR_TIMEOUT = -6
BC_ERR_BOUNDS = -7
BC_ERR_UNSUPPORTED = -8
BC_ERR_STATE = -9

BC_STATUS_SIGMA_OVERFLOW = 0x1
BC_STATUS_DENSE_TIMEOUT = 0x8
BC_STATUS_COPY_TIMEOUT = 0x10

BC_GRAPH_TRUST_INPUT = 0x1
BC_GRAPH_DIRECTED = 0x2

BC_HALVE = 0x1
BC_ACCUMULATE = 0x2
BC_PLAIN = 0x4
BC_TIMING = 0x8
BC_NO_HASH = 0x10
BC_DENSE = 0x20
BC_SPARSE_BACKWARD = 0x40
BC_KEEP_ORDER = 0x80
BC_PAIRS = 0x100
BC_TEST_WAIT_EXPIRY = 0x200
BC_FORCE_BOTTOMUP = 0x400

BC_KERNEL_INIT = 0
BC_KERNEL_FORWARD = 1
BC_KERNEL_BACKWARD = 2
BC_KERNEL_HASH = 3
BC_KERNEL_PLAIN = 4
BC_KERNEL_DENSE = 5
KERNEL_NAMES = {0: "init", 1: "forward", 2: "backward", 3: "hash", 4: "plain", 5: "dense"}

# every entry point include/bc_gb300.h declares
EXPORTS = ["bc_create_graph", "bc_run", "bc_result", "bc_source_hashes", "bc_forward_rows",
           "bc_kernel_time", "bc_kernel_trace", "bc_run_stats", "bc_launch_count", "bc_graph_size", "bc_destroy_graph",
           "bc_release_cached_memory", "bc_vertex_order",
           "bc_status_string", "bc_last_error", "bc_run_noalloc", "bc_autotune", "bc_set_default_options",
           "bc_last_options",
           "bc_many_create", "bc_many_run", "bc_many_result", "bc_many_stats", "bc_many_destroy", "bc_run_many"]


class BcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: status {code} ({msg})")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("flags", ctypes.c_uint32), ("chunk", ctypes.c_int32),
                ("delta", ctypes.c_int32), ("wait_limit_ms", ctypes.c_int64),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("device_wait_us", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("reserved1", ctypes.c_int64 * 2)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True, require_gpu: bool = True):
    """Load the shared library (building it first when stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        lib = ctypes.CDLL(_build.LIB)
        P = ctypes.c_void_p
        i32, u32, i64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64
        sig = {
            "bc_create_graph": (i32, [i32, P, P, P, u32, ctypes.POINTER(P)]),
            "bc_run": (i32, [P, P, i32, P, P]),
            "bc_result": (i32, [P, P, P]),
            "bc_source_hashes": (i32, [P, P, P, P, P]),
            "bc_forward_rows": (i32, [P, P, i32, P, P, P, P]),
            "bc_kernel_time": (i32, [P, i32, P, P]),
            "bc_kernel_trace": (i32, [P, i64, P, P, P, P]),
            "bc_run_stats": (i32, [P, P, P, P, P]),
            "bc_launch_count": (i64, [P]),
            "bc_graph_size": (i32, [P, P, P, P]),
            "bc_destroy_graph": (None, [P]),
            "bc_release_cached_memory": (None, []),
            "bc_vertex_order": (i32, [i32, P, P, P]),
            "bc_status_string": (ctypes.c_char_p, [i32]),
            "bc_last_error": (ctypes.c_char_p, []),
            "bc_run_noalloc": (i32, [i32, P, P, P, i32, P, P]),
            "bc_autotune": (i32, [P, i32, P, P]),
            "bc_set_default_options": (i32, [P, P]),
            "bc_last_options": (i32, [P, P]),
            "bc_many_create": (i32, [P, i32, P, ctypes.POINTER(P)]),
            "bc_many_run": (i32, [P, P]),
            "bc_many_result": (i32, [P, P, P]),
            "bc_many_stats": (i32, [P, P]),
            "bc_many_destroy": (None, [P]),
            "bc_run_many": (i32, [P, i32, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if require_gpu:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device visible: the betweenness library has no CPU path")
            torch.cuda.init()
        _lib = lib
    return _lib


def _check(code: int, where: str, allow_warn: bool = True) -> int:
    if code == BC_OK or (allow_warn and code == BC_WARN_SIGMA_OVERFLOW):
        return code
    lib = load(require_gpu=False)
    msg = lib.bc_last_error().decode() or lib.bc_status_string(code).decode()
    raise BcError(code, where, msg)


def _addr(x):
    """Pointer of a numpy array or a torch tensor (host or device); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_options(batch=0, flags=0, chunk=0, wait_limit_ms=0, alpha=0.0, beta=0.0, delta=0,
                 device_wait_us=0) -> Options:
    o = Options()
    o.batch, o.flags, o.chunk, o.wait_limit_ms = batch, flags, chunk, wait_limit_ms
    o.alpha, o.beta, o.delta, o.device_wait_us = alpha, beta, delta, device_wait_us
    return o


class Graph:
    """A graph handle of the library (bc_create_graph ... bc_destroy_graph).

    row_ptr / col / weights may be numpy arrays (host) or torch tensors
    (host or CUDA), int32, C-contiguous.
    """

    def __init__(self, n: int, row_ptr, col, weights=None, trust_input: bool = False, directed: bool = False):
        self.lib = load()
        h = ctypes.c_void_p()
        flags = (BC_GRAPH_TRUST_INPUT if trust_input else 0) | (BC_GRAPH_DIRECTED if directed else 0)
        for a in (row_ptr, col, weights):
            if a is not None and getattr(a, "dtype", None) not in (np.int32, None) and str(a.dtype) != "torch.int32":
                raise TypeError("CSR arrays must be int32")
        _check(self.lib.bc_create_graph(int(n), _addr(row_ptr), _addr(col), _addr(weights), flags,
                                        ctypes.byref(h)), "bc_create_graph", allow_warn=False)
        self.handle = h
        self.n = int(n)

    @classmethod
    def from_csr(cls, g, **kw):
        kw.setdefault("directed", bool(getattr(g, "directed", False)))
        return cls(g.n, np.ascontiguousarray(g.row_ptr, np.int32), np.ascontiguousarray(g.col, np.int32),
                   None if g.w is None else np.ascontiguousarray(g.w, np.int32), **kw)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bc_destroy_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, sources=None, batch=0, flags=0, chunk=0, wait_limit_ms=0, stream=None, alpha=0.0, beta=0.0,
            delta=0, device_wait_us=0, default_options=False) -> int:
        """bc_run: sources None = all vertices; numpy int32 (host) or torch int32 (host/device).
        default_options=True passes NULL options (the library's defaults or its tuned choice)."""
        opt = make_options(batch, flags, chunk, wait_limit_ms, alpha, beta, delta, device_wait_us)
        if sources is not None and isinstance(sources, np.ndarray):
            sources = np.ascontiguousarray(sources, dtype=np.int32)
        ns = 0 if sources is None else int(len(sources))
        return _check(self.lib.bc_run(self.handle, _addr(sources), ns, None if default_options else ctypes.byref(opt),
                                      _stream_ptr(stream)), "bc_run")

    def result(self, out=None):
        """bc_result into `out` (numpy float64 / torch float64 host or device); returns (out, status, flags)."""
        if out is None:
            out = np.empty(self.n, np.float64)
        fl = ctypes.c_uint32(0)
        code = _check(self.lib.bc_result(self.handle, _addr(out), ctypes.byref(fl)), "bc_result")
        return out, code, fl.value

    def source_hashes(self, k: int):
        hs = np.empty(k, np.uint64)
        hd = np.empty(k, np.uint64)
        ds = np.empty(k, np.int64)
        rc = np.empty(k, np.int64)
        _check(self.lib.bc_source_hashes(self.handle, _addr(hs), _addr(hd), _addr(ds), _addr(rc)),
               "bc_source_hashes")
        return dict(hash_sigma=hs, hash_dist=hd, dist_sum=ds, reach=rc)

    def forward_rows(self, sources, batch=0, stream=None, flags=0):
        src = np.ascontiguousarray(sources, dtype=np.int32)
        k = int(src.size)
        sig = np.empty((k, self.n), np.uint64)
        dist = np.empty((k, self.n), np.int32)
        opt = make_options(batch, flags)
        code = _check(self.lib.bc_forward_rows(self.handle, _addr(src), k, _addr(sig), _addr(dist),
                                               ctypes.byref(opt), _stream_ptr(stream)), "bc_forward_rows")
        return sig, dist, code

    def kernel_time(self, kind: int):
        n = ctypes.c_int64(0)
        t = ctypes.c_double(0.0)
        _check(self.lib.bc_kernel_time(self.handle, kind, ctypes.byref(n), ctypes.byref(t)), "bc_kernel_time")
        return n.value, t.value

    def kernel_trace(self):
        """bc_kernel_trace: (kind, level, ms) arrays of every launch of the last BC_TIMING run."""
        cnt = ctypes.c_int64(0)
        _check(self.lib.bc_kernel_trace(self.handle, 0, None, None, None, ctypes.byref(cnt)), "bc_kernel_trace")
        k = cnt.value
        kind = np.empty(k, np.int32)
        level = np.empty(k, np.int32)
        ms = np.empty(k, np.float32)
        _check(self.lib.bc_kernel_trace(self.handle, k, _addr(kind), _addr(level), _addr(ms), ctypes.byref(cnt)),
               "bc_kernel_trace")
        return kind, level, ms

    def autotune(self, sample: int = 0, stream=None) -> Options:
        """bc_autotune: time the candidates on `sample` sources; the choice
        becomes this handle's default for run(default_options=True)."""
        o = Options()
        _check(self.lib.bc_autotune(self.handle, int(sample), ctypes.byref(o), _stream_ptr(stream)), "bc_autotune")
        return o

    def set_default_options(self, opt) -> None:
        _check(self.lib.bc_set_default_options(self.handle, None if opt is None else ctypes.byref(opt)),
               "bc_set_default_options")

    def last_options(self) -> Options:
        o = Options()
        _check(self.lib.bc_last_options(self.handle, ctypes.byref(o)), "bc_last_options")
        return o

    def run_stats(self):
        a = ctypes.c_int64(0)
        d = ctypes.c_int64(0)
        _check(self.lib.bc_run_stats(self.handle, ctypes.byref(a), ctypes.byref(d), None, None), "bc_run_stats")
        return a.value, d.value

    def dense_flops(self) -> float:
        """Tensor-core work of the last BC_DENSE run, bf16 and e4m3 together."""
        bf, f8 = self.dense_flops_by_type()
        return bf + f8

    def dense_flops_by_type(self):
        """(bf16 flops, e4m3 flops) of the last BC_DENSE run."""
        f = ctypes.c_double(0.0)
        f8 = ctypes.c_double(0.0)
        _check(self.lib.bc_run_stats(self.handle, None, None, ctypes.byref(f), ctypes.byref(f8)), "bc_run_stats")
        return f.value, f8.value

    def launch_count(self) -> int:
        return int(self.lib.bc_launch_count(self.handle))


class ManyPlan:
    """bc_many_create / bc_many_run / bc_many_result over Graph handles: all
    sources of every graph in one persistent launch replayed from a CUDA graph."""

    def __init__(self, graphs, batch: int = 32):
        self.lib = load()
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle.value for g in self.graphs])
        self._arr = arr
        h = ctypes.c_void_p()
        opt = make_options(batch)
        _check(self.lib.bc_many_create(arr, len(self.graphs), ctypes.byref(opt), ctypes.byref(h)),
               "bc_many_create", allow_warn=False)
        self.handle = h

    def run(self, stream=None):
        _check(self.lib.bc_many_run(self.handle, _stream_ptr(stream)), "bc_many_run")

    def result(self):
        fl = ctypes.c_uint32(0)
        rr = ctypes.c_int32(0)
        code = _check(self.lib.bc_many_result(self.handle, ctypes.byref(fl), ctypes.byref(rr)), "bc_many_result")
        return code, fl.value, rr.value

    def dag_arcs(self) -> int:
        a = ctypes.c_int64(0)
        _check(self.lib.bc_many_stats(self.handle, ctypes.byref(a)), "bc_many_stats")
        return a.value

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bc_many_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def release_cached_memory() -> None:
    """Free the device blocks kept from destroyed graph handles."""
    load().bc_release_cached_memory()


def vertex_order(n: int, row_ptr, col) -> np.ndarray:
    """bc_vertex_order: perm[v] = v's id in the numbering with locality that the
    weighted sweep runs on (host code; no GPU needed)."""
    _build.build()
    lib = ctypes.CDLL(_build.LIB)  # a host-only call: not the cached handle, which demands a GPU
    lib.bc_vertex_order.restype = ctypes.c_int32
    lib.bc_vertex_order.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    perm = np.empty(max(n, 0), dtype=np.int32)
    code = lib.bc_vertex_order(int(n), _addr(rp), _addr(cl) if cl.size else None, _addr(perm))
    if code != BC_OK:
        lib.bc_last_error.restype = ctypes.c_char_p
        raise BcError(code, "bc_vertex_order", lib.bc_last_error().decode())
    return perm


def betweenness(g, sources=None, batch=0, flags=0, stream=None):
    """One-call helper: upload, run, read back. Returns (bc float64[n], status)."""
    with Graph.from_csr(g) as h:
        h.run(sources, batch=batch, flags=flags, stream=stream)
        out, code, _ = h.result()
        return out, code
