"""CPU oracle for exact betweenness centrality -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package. The GPU library shares no code with it
and never calls it.

Three independent routes to the same numbers (Kintali, "Betweenness
Centrality: Algorithms and Lower Bounds"):

* :func:`bc` / :func:`source` -- textbook Brandes (Section 1.1, Theorem 1.1)
  in plain C (``brandes.c``): BFS or binary-heap Dijkstra, 128-bit path counts,
  FP64 dependencies.
* :mod:`oracle.brute` -- the definitions of Section 1.1 by enumeration of
  every shortest path (pure Python, exact fractions; tiny graphs).
* :mod:`oracle.algebraic` -- Section 3.1's matrix forms (ComputePathCount,
  ComputeDependency; the path-count mask read as "not reached yet") and
  Algorithm 2's pair formula (Section 4.2.1), in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OVERFLOW64 = 1
OVERFLOW128 = 2
BAD_INPUT = 4
OOM = 8


def build(force: bool = False) -> str:
    """Compile brandes.c with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32 = ctypes.c_int32
            lib.oracle_source.restype = i32
            lib.oracle_source.argtypes = [i32, P, P, P, P, P, P, i32, P, P, P, P, P, P, P]
            lib.oracle_bc.restype = i32
            lib.oracle_bc.argtypes = [i32, P, P, P, P, P, P, P, i32, i32, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.int32)
    return rp, col, w


def _in_csr(g):
    """In-arc CSR of a directed graph (its transpose), or Nones: an undirected
    graph's out-arcs serve as in-arcs."""
    if not getattr(g, "directed", False):
        return None, None, None
    from paper_0809_1906_gb300.graphs import transpose
    return _csr(transpose(g))


def source(g, s: int, with_delta: bool = True) -> dict:
    """Full forward (and backward) rows for one source.

    Returns dist (int64, -1 unreachable), sigma (uint64, count mod 2^64),
    sigma_hi (uint64, bits 64..127), delta (float64, delta_s*(v); delta[s] is
    reach-1), order (settle order), reach, arcs (shortest-path DAG arcs),
    flags (OVERFLOW64 when some count >= 2^64).
    """
    lib = _load()
    rp, col, w = _csr(g)
    n = g.n
    dist = np.empty(n, np.int64)
    lo = np.empty(n, np.uint64)
    hi = np.empty(n, np.uint64)
    delta = np.empty(n, np.float64) if with_delta else None
    order = np.empty(max(n, 1), np.int32)
    flags = ctypes.c_int32(0)
    arcs = ctypes.c_int64(0)
    irp, icol, iw = _in_csr(g)
    cnt = lib.oracle_source(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(irp), _ptr(icol), _ptr(iw), int(s),
                            _ptr(dist), _ptr(lo), _ptr(hi),
                            _ptr(delta), _ptr(order), ctypes.byref(flags), ctypes.byref(arcs))
    if cnt < 0:
        raise ValueError(f"oracle_source rejected input (flags={flags.value})")
    return dict(dist=dist, sigma=lo, sigma_hi=hi, delta=delta, order=order[:cnt], reach=cnt,
                arcs=arcs.value, flags=flags.value)


def bc(g, sources=None, threads: int = 0) -> dict:
    """Ordered-pair betweenness over `sources` (None = all vertices).

    Returns bc (float64[n]) and per-source hash_sigma, hash_dist (uint64),
    dist_sum, reach, arcs (int64) in source-list order, plus flags.
    """
    lib = _load()
    rp, col, w = _csr(g)
    n = g.n
    src = None if sources is None else np.ascontiguousarray(sources, dtype=np.int32)
    ns = n if src is None else int(src.size)
    out = np.zeros(n, np.float64)
    hs = np.zeros(ns, np.uint64)
    hd = np.zeros(ns, np.uint64)
    ds = np.zeros(ns, np.int64)
    rc = np.zeros(ns, np.int64)
    ar = np.zeros(ns, np.int64)
    flags = ctypes.c_int32(0)
    irp, icol, iw = _in_csr(g)
    r = lib.oracle_bc(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(irp), _ptr(icol), _ptr(iw), _ptr(src), ns,
                      int(threads), _ptr(out),
                      _ptr(hs), _ptr(hd), _ptr(ds), _ptr(rc), _ptr(ar), ctypes.byref(flags))
    if r != 0:
        raise ValueError(f"oracle_bc rejected input (flags={flags.value})")
    return dict(bc=out, hash_sigma=hs, hash_dist=hd, dist_sum=ds, reach=rc, arcs=ar, flags=flags.value)
