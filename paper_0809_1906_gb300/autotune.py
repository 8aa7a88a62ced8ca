"""Autotuner for the launch parameters of the batched paths.

For one graph the library's own tuner (bc_autotune) times bc_run on a sample
of sources with CUDA events: unweighted graphs, every batch width (sources
per batch: 64, 128, 256) x work-item chunk size (arcs per warp item before a
high-degree vertex is split: 128, 256, 512), then the look-ahead's tail
threshold beta (1/256, 1/64, 1/16); weighted graphs, the wave size.
The choice becomes the handle's default, which bc_run uses when it is given
no options. Here it is also cached in a JSON file keyed by (n, m,
degree-skew bucket, GPU name), so a graph of the same shape on the same GPU
gets it installed (bc_set_default_options) without timing again.

For a many-graph plan it times the persistent launch for batch widths 32, 64,
128 and 256 and keeps the fastest.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import numpy as np

from . import graphs as G
from . import native

CACHE = os.environ.get("BCGB_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))


def _key(g, kind: str) -> str:
    import torch
    deg = g.degrees()
    skew = int(round(math.log2(max(1.0, deg.max() / max(deg.mean(), 1e-9))))) if deg.size else 0
    n_b = int(round(math.log2(max(g.n, 1))))
    m_b = int(round(math.log2(max(g.m, 1))))
    return f"{kind}|n2^{n_b}|m2^{m_b}|skew{skew}|w{int(g.weighted)}|{torch.cuda.get_device_name()}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time_ms(fn, reps=2):
    import torch
    stream = torch.cuda.current_stream()
    fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_graph(g, handle=None, sample=2048, use_cache=True):
    """Best launch options for bc_run on graph g, installed as the handle's
    default. Returns a dict with batch, chunk, alpha, beta (and whether it
    came from the cache)."""
    key = _key(g, "graph")
    cache = _load()
    own = handle is None
    h = handle or native.Graph.from_csr(g, trust_input=True)
    try:
        if use_cache and key in cache:
            c = cache[key]
            h.set_default_options(native.make_options(c["batch"], 0, c["chunk"], alpha=c["alpha"], beta=c["beta"]))
            return dict(c, cached=True)
        o = h.autotune(sample)
        out = {"batch": int(o.batch), "chunk": int(o.chunk), "alpha": float(o.alpha), "beta": float(o.beta)}
    finally:
        if own:
            h.close()
    cache = _load()
    cache[key] = out
    _store(cache)
    return dict(out, cached=False)


def tune_many(gs, handles, batches=(32, 64, 128, 256), use_cache=True):
    """Best batch width for a many-graph plan over handles."""
    big = max(gs, key=lambda g: g.n * g.m)
    key = _key(big, f"many{len(gs)}")
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    res = {}
    for b in batches:
        with native.ManyPlan(handles, batch=b) as plan:
            res[str(b)] = _time_ms(lambda: (plan.run(), plan.result()))
    best = int(min(res, key=res.get))
    out = {"batch": best, "ms": res}
    cache = _load()
    cache[key] = out
    _store(cache)
    return out
