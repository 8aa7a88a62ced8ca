"""Benchmark: exact betweenness centrality, BC edges/s (sources x m / s).

Default workload: R-MAT scale 16, edge factor 16, (a,b,c,d) =
(0.57,0.19,0.19,0.05), symmetrised, largest connected component; every LCC
vertex is a source, batches of 256. One step = one bc_run over all sources
plus its device-side result (the whole hot path: batch init, forward
counting, backward sweep with the FP64 BC reduction, per-source summaries).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). The roofline numerator is the algorithmic
bytes of Brandes per source (algorithmic_bytes below) divided by the
kernels' CUDA-event time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0809_1906_gb300 import graphs as G  # noqa: E402

METRIC = "BC edges/sec (sources x m / s)"
UNIT = "edges/s"
BATCH = 256


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# Sources of the sweep kernels whose DRAM bytes profiles/traffic_rmat.json holds.
SWEEP_SOURCES = ("msbfs.cu", "msbfs_body.cuh", "rowstage.cuh", "pdl.cuh", "bc_internal.cuh")


def code_text(text: str) -> str:
    """A C/CUDA source with its comments and blank space removed."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "".join(text.split())


# Sources of the weighted kernel whose DRAM bytes profiles/traffic_grid.json holds.
GRID_SOURCES = ("sssp_packed.cu", "weighted.cuh", "relabel.cu")


def csrc_digest(names=SWEEP_SOURCES) -> str:
    """SHA-256 over the kernels' sources with comments and blank space
    removed: DRAM counters taken from an older build do not describe the
    current kernels, while a comment edit changes nothing they measure."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_0809_1906_gb300", "csrc", name), encoding="utf-8") as fh:
            h.update(name.encode())
            h.update(code_text(fh.read()).encode())
    return h.hexdigest()


# Kernel kinds of bc_kernel_time and the kernels each one times.
KIND_KERNELS = {"init": ("k_init",), "forward": ("k_first", "k_forward"), "backward": ("k_backward",),
                "hash": ("k_hash",)}
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic_rmat.json")


def measured_traffic(kind: str, path: str = TRAFFIC_JSON):
    """DRAM bytes (read + write) per launch of kernel kind `kind`, from the
    committed ncu capture of one 256-source batch (profiles/traffic_rmat.json);
    None when the capture was taken on other kernel sources."""
    try:
        with open(path) as f:
            tr = json.load(f)
        if tr.get("csrc_sha256") != csrc_digest():
            return None
        return tr["kinds"][kind]["dram_bytes_per_launch"]
    except Exception:
        return None


def write_traffic(csv_path: str, command: str, out_path: str = TRAFFIC_JSON, echo: bool = True):
    """Turn an ncu capture (metrics dram__bytes_read.sum, dram__bytes_write.sum,
    gpu__time_duration.sum; --csv) of one batch of the R-MAT workload into
    profiles/traffic_rmat.json: per kernel kind, the DRAM bytes of that batch's
    launches (the 256-wide kernels only; the landmark pass runs 32-wide) divided
    by their number."""
    import collections
    import csv
    with open(csv_path) as f:
        rows = list(csv.reader(line for line in f if line.startswith('"')))
    h = rows[0]
    per = collections.defaultdict(dict)
    for r in rows[1:]:
        i = int(r[h.index("ID")])
        name = r[h.index("Kernel Name")].split("(")[0].split("::")[-1]
        per[i]["kernel"] = name.split("<")[0]
        per[i]["wide"] = name.startswith(per[i]["kernel"] + "<8")
        per[i][r[h.index("Metric Name")]] = float(r[h.index("Metric Value")].replace(",", ""))
    kinds = {}
    for kind, names in KIND_KERNELS.items():
        sel = [x for x in per.values() if x["kernel"] in names and x["wide"]]
        if not sel:
            continue
        rd = sum(x.get("dram__bytes_read.sum", 0.0) for x in sel)
        wr = sum(x.get("dram__bytes_write.sum", 0.0) for x in sel)
        kinds[kind] = {"launches": len(sel), "dram_bytes_per_launch": (rd + wr) / len(sel), "dram_read_bytes": rd,
                       "dram_write_bytes": wr,
                       "ncu_time_ms": sum(x.get("gpu__time_duration.sum", 0.0) for x in sel) / 1e6}
    out = {"csrc_sha256": csrc_digest(), "command": command,
           "note": "one 256-source batch of the R-MAT workload (seeded sample, one lane); ncu replays each launch "
                   "with cold caches, so bytes are an upper bound of a warm run; per launch of each kind",
           "kinds": kinds}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    if echo:
        print(json.dumps(out, indent=1))
    return out


TRAFFIC_GRID_JSON = os.path.join(ROOT, "profiles", "traffic_grid.json")


def measured_traffic_grid(path: str = TRAFFIC_GRID_JSON):
    """DRAM bytes (read + write) per source of k_wsssp_packed on the weighted
    grid, from the committed ncu capture of one wave
    (profiles/traffic_grid.json); None when taken on other kernel sources."""
    try:
        with open(path) as f:
            tr = json.load(f)
        if tr.get("csrc_sha256") != csrc_digest(GRID_SOURCES):
            return None
        return tr["dram_bytes_per_source"]
    except Exception:
        return None


def write_traffic_grid(csv_path: str, sources: int, command: str, out_path: str = TRAFFIC_GRID_JSON):
    """Turn an ncu capture (dram__bytes_read.sum, dram__bytes_write.sum,
    gpu__time_duration.sum; --csv) of k_wsssp_packed launches over `sources`
    sources of the weighted grid into profiles/traffic_grid.json."""
    import csv
    with open(csv_path) as f:
        rows = list(csv.reader(line for line in f if line.startswith('"')))
    h = rows[0]
    tot = {}
    ids = set()
    for r in rows[1:]:
        if "k_wsssp_packed" not in r[h.index("Kernel Name")]:
            continue
        ids.add(r[h.index("ID")])
        k = r[h.index("Metric Name")]
        tot[k] = tot.get(k, 0.0) + float(r[h.index("Metric Value")].replace(",", ""))
    rd, wr = tot.get("dram__bytes_read.sum", 0.0), tot.get("dram__bytes_write.sum", 0.0)
    out = {"csrc_sha256": csrc_digest(GRID_SOURCES), "command": command,
           "note": "k_wsssp_packed over one wave of the weighted grid's seeded sources (relabelled graph); ncu "
                   "replays the launch with cold caches; bytes per source = (read + write) / sources",
           "launches": len(ids), "sources": sources, "dram_read_bytes": rd, "dram_write_bytes": wr,
           "dram_bytes_per_source": (rd + wr) / max(sources, 1),
           "ncu_time_ms": tot.get("gpu__time_duration.sum", 0.0) / 1e6}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))
    return out


def workload():
    g = G.rmat_lcc(16, 16)
    return g, f"rmat_s16_ef16_lcc (n={g.n}, m={g.m}), all {g.n} sources, batch {BATCH}"


def algorithmic_bytes(n, m, arcs_total, nsrc, B):
    """Bytes Brandes must move, per pass (one look per arc per pass):
    forward  2m x 1 B level probe + 8 B sigma x a + 9 B (sigma + level) x n
    backward 2m x 1 B level probe + 4 B c x a + 13 B (sigma + level read, c write) x n
    per batch: BC 16 B x n, CSR 2 x (8m + 4n) B (read by each pass)."""
    nb = -(-nsrc // B)
    fwd = nsrc * (2 * m + 9 * n) + 8 * arcs_total + nb * (8 * m + 4 * n)
    bwd = nsrc * (2 * m + 13 * n) + 4 * arcs_total + nb * (8 * m + 4 * n + 16 * n)
    return fwd, bwd


def cpu_oracle_rate(g, seconds: float):
    """Oracle (as it stands) on the host cores over a bounded sample of sources."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    probe = G.sample_sources(g.n, min(g.n, 2 * threads), 901)
    t0 = time.perf_counter()
    oracle.bc(g, probe, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    k = int(min(g.n, max(len(probe), len(probe) * seconds / dt)))
    src = G.sample_sources(g.n, k, 902)
    t0 = time.perf_counter()
    oracle.bc(g, src, threads=threads)
    dt = time.perf_counter() - t0
    return k * g.m / dt, threads, k, dt


def run_reference(args, rank):
    if rank != 0:
        return
    g, desc = workload()
    per_step = max(2.0, 20.0 / max(args.steps, 1))
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, k, dt = cpu_oracle_rate(g, per_step if i >= args.warmup else 1.0)
        if i >= args.warmup:
            vals.append((v, k, dt))
    v = statistics.median([x[0] for x in vals])
    ms = 1000.0 * statistics.median([x[2] / x[1] * g.n for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u128+f64", "data": "synthetic",
            "config": {"workload": desc, "n": g.n, "m": g.m, "sources": g.n, "batch": BATCH},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{vals[0][1]} seeded sources per step (bounded sample of the all-sources job); "
                                       "ms_per_step extrapolated to all sources"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(fn, steps, warmup, stream, flush):
    """Median CUDA-event time (ms) of fn() on `stream`, L2 flushed before each step."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _oracle_rate(g, sources, seconds):
    """Oracle edges/s on a bounded prefix of `sources` (all host cores)."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    k = min(len(sources), 2 * threads)
    t0 = time.perf_counter()
    oracle.bc(g, sources[:k], threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    k = int(min(len(sources), max(k, k * seconds / dt)))
    t0 = time.perf_counter()
    oracle.bc(g, sources[:k], threads=threads)
    dt = time.perf_counter() - t0
    return {"value": k * g.m / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{k} of the workload's sources ({dt:.1f} s)"}


def err_stats(got, ref, n, what):
    """Error of a device BC vector against the FP64 oracle over the same
    sources: the largest relative error where the relative bound 1e-5 |ref|
    is the binding one (|ref| >= 0.1 n), the largest absolute error
    elsewhere (bound 1e-6 n), and whether every vertex is within
    max(1e-5 |ref|, 1e-6 n)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * max(n, 1))
    rel = np.abs(ref) >= 0.1 * max(n, 1)
    return {"max_rel_err": float(np.max(err[rel] / np.abs(ref[rel]))) if rel.any() else 0.0,
            "max_abs_err_small_ref": float(np.max(err[~rel])) if (~rel).any() else 0.0,
            "within_tolerance": bool(np.all(err <= tol)), "sample": what}


class Ctx:
    """What every configuration's measurement shares: the stream, the L2
    flush buffer, the step counts and the CPU-time budget of the oracle."""

    def __init__(self, args, cpu_seconds):
        import torch
        from paper_0809_1906_gb300 import native
        native.load()
        self.native = native
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        self.steps, self.warmup = args.steps, args.warmup
        self.cpu_seconds = cpu_seconds
        self.hbm, self.hbm_kind = peaks()

    def timed(self, fn, steps=None, warmup=None):
        return _timed(fn, steps or self.steps, warmup or self.warmup, self.stream, self.flush)


def cfg_er1024(c):
    """ER n=1024 + Hamiltonian path, all sources (launch/latency bound)."""
    import torch
    nat = c.native
    g = G.er_hamiltonian()
    src = torch.arange(g.n, dtype=torch.int32, device="cuda")
    import oracle
    ref = oracle.bc(g)["bc"]
    with nat.Graph.from_csr(g) as h:
        res = {}
        for b in (32, 64, 128, 256):
            res[b] = c.timed(lambda: (h.run(src, batch=b, stream=c.stream), h.result()))
        best = min(res, key=res.get)
        h.run(src, batch=best, stream=c.stream)
        got, _, _ = h.result()
        ms_plain = c.timed(lambda: (h.run(src, flags=nat.BC_PLAIN, stream=c.stream), h.result()), 2, 1)
    return {"metric": METRIC, "unit": UNIT, "value": g.n * g.m / (res[best] / 1e3), "ms_per_step": res[best],
            "config": {"workload": f"ER n={g.n} m={g.m} + Hamiltonian path, all sources", "batch": best,
                       "ms_by_batch": res},
            "roofline": None, "roofline_note": "launch/latency bound: 5.2M source-edges per step",
            "vs_plain_gpu": {"value": g.n * g.m / (ms_plain / 1e3), "ms": ms_plain, "speedup": ms_plain / res[best]},
            "error_vs_oracle": err_stats(got, ref, g.n, "all sources"),
            "cpu_baseline": _oracle_rate(g, np.arange(g.n, dtype=np.int32), c.cpu_seconds)}


def cfg_grid(c):
    """512x512 grid + 5% long-range edges, integer weights U[1,100]: 4096
    sampled sources (integer buckets with tie-aware counts), plus the 64x64
    subgrid over all sources."""
    import torch
    import oracle
    nat = c.native
    g = G.grid_longrange()
    srcn = G.sample_sources(g.n, 4096, 33)
    src = torch.from_numpy(srcn).cuda()
    with nat.Graph.from_csr(g) as h:
        ms = c.timed(lambda: (h.run(src, stream=c.stream), h.result()))
        arcs, _ = h.run_stats()
        h.run(src, flags=nat.BC_TIMING, stream=c.stream)
        h.result()
        fl, fms = h.kernel_time(nat.BC_KERNEL_FORWARD)
        esrc = srcn[:256]
        h.run(esrc, stream=c.stream)
        got, _, _ = h.result()
    err = err_stats(got, oracle.bc(g, esrc)["bc"], g.n, "256 of the 4096 sampled sources")
    sub = G.induced_subgrid(g, 512, 64)
    with nat.Graph.from_csr(sub) as hs:
        ms_sub = c.timed(lambda: (hs.run(stream=c.stream), hs.result()))
        gsub, _, _ = hs.result()
    err_sub = err_stats(gsub, oracle.bc(sub)["bc"], sub.n, "64x64 subgrid, all sources")
    n, m = g.n, g.m
    alg = 4096 * (16 * m + 32 * n) + 12 * arcs  # per source: 2 passes x 2m x 4 B, 12 B per DAG arc, 32 B per vertex
    achieved = alg / (fms / 1e3) / 1e9
    tps = measured_traffic_grid()  # DRAM bytes per source, scaled to the sources of an average launch
    traffic = tps * 4096 / max(fl, 1) if tps is not None else None
    return {"metric": METRIC, "unit": UNIT, "value": 4096 * m / (ms / 1e3), "ms_per_step": ms,
            "config": {"workload": f"512x512 grid + 5% long-range, w~U[1,100] (n={n}, m={m}), 4096 sampled sources",
                       "dag_arcs_per_source": arcs / 4096,
                       "subgrid64_all_sources": {"n": sub.n, "m": sub.m, "ms": ms_sub,
                                                 "value": sub.n * sub.m / (ms_sub / 1e3),
                                                 "error_vs_oracle": err_sub}},
            "roofline": {"bound": "hbm", "kernel": "k_wsssp_packed", "achieved": achieved, "peak": c.hbm,
                         "unit": "GB/s", "frac": achieved / c.hbm, "peak_source": c.hbm_kind, "traffic": traffic,
                         "traffic_note": "profiles/traffic_grid.json: DRAM bytes per source x sources per launch",
                         "algorithmic_bytes": alg, "kernel_ms": fms, "launches": fl},
            "error_vs_oracle": err,
            "cpu_baseline": _oracle_rate(g, srcn, c.cpu_seconds)}


def cfg_gnp(c, full=False):
    """G(8192, 0.05), all sources, the algebraic form on tensor cores (BC_DENSE)."""
    import torch
    import oracle
    nat = c.native
    g = G.gnp(8192, 0.05)
    src = torch.arange(g.n, dtype=torch.int32, device="cuda")
    with nat.Graph.from_csr(g) as h:
        ms_d = c.timed(lambda: (h.run(src, flags=nat.BC_DENSE, stream=c.stream), h.result()))
        h.run(src, flags=nat.BC_DENSE | nat.BC_TIMING, stream=c.stream)
        h.result()
        kinds = {nat.KERNEL_NAMES[k]: h.kernel_time(k) for k in nat.KERNEL_NAMES}
        fl16, fl8 = h.dense_flops_by_type()
        flops = fl16 + fl8
        ms_s = {b: c.timed(lambda: (h.run(src, batch=b, stream=c.stream), h.result()), 2, 1)
                for b in ((128, 256) if full else (256,))}
        esrc = G.sample_sources(g.n, 512, 61)
        h.run(esrc, flags=nat.BC_DENSE, stream=c.stream)
        got, _, _ = h.result()
    err = err_stats(got, oracle.bc(g, esrc)["bc"], g.n, "512 seeded sources, BC_DENSE")
    dn, dms = kinds["dense"]
    tf = flops / (dms / 1e3) / 1e12 if dms else 0.0
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        bf16 = float(json.load(f)["bf16_tflops"])
    # e4m3 runs at twice the bf16 rate (nominal 4.5 against 2.25 PFLOP/s): the
    # peak of the mix is the flop-weighted harmonic one, so frac is the share
    # of the time the tensor pipe at its peak rates would need
    f8 = 2.0 * bf16
    peak = flops / (fl16 / bf16 + fl8 / f8) if flops else bf16
    return {"metric": METRIC, "unit": UNIT, "value": g.n * g.m / (ms_d / 1e3), "ms_per_step": ms_d,
            "config": {"workload": f"G(n=8192, p=0.05) (m={g.m}), all sources, 64 batches of 128, BC_DENSE",
                       "kernels_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in kinds.items()}},
            "roofline": {"bound": "tensor", "kernel": "k_dense_level", "achieved": tf, "peak": peak,
                         "unit": "TFLOP/s", "frac": tf / peak,
                         "peak_source": "measured bf16 burst; e4m3 at 2x (nominal ratio), weighted by flops",
                         "flops": flops, "flops_bf16": fl16, "flops_e4m3": fl8, "traffic": None},
            "vs_sparse_same_graph": {str(b): {"ms": v, "value": g.n * g.m / (v / 1e3), "speedup": v / ms_d}
                                     for b, v in ms_s.items()},
            "error_vs_oracle": err,
            "cpu_baseline": _oracle_rate(g, np.arange(g.n, dtype=np.int32), c.cpu_seconds)}


def cfg_many(c):
    """2000 graphs, n log-uniform in [50, 5000], all sources of every graph in
    one persistent launch replayed from a captured CUDA graph."""
    import oracle
    nat = c.native
    gs = G.many_graphs()
    hs = [nat.Graph.from_csr(g, trust_input=True) for g in gs]
    work = float(sum(g.n * g.m for g in gs))
    from paper_0809_1906_gb300 import autotune
    best = autotune.tune_many(gs, hs)["batch"]
    pick = np.random.default_rng(20080919).choice(len(gs), 40, replace=False)
    with nat.ManyPlan(hs, batch=best) as plan:
        def step():
            plan.run(c.stream)
            plan.result()
        ms = c.timed(step)
        arcs = plan.dag_arcs()
        errs = [err_stats(hs[i].result()[0], oracle.bc(gs[i])["bc"], gs[i].n, "") for i in pick.tolist()]
    for h in hs:
        h.close()
    err = {"max_rel_err": max(e["max_rel_err"] for e in errs),
           "max_abs_err_small_ref": max(e["max_abs_err_small_ref"] for e in errs),
           "within_tolerance": all(e["within_tolerance"] for e in errs),
           "sample": "40 seeded graphs of the set, all sources each"}
    # algorithmic bytes: per source 4m + 22n, plus 12 B per DAG arc
    alg = float(sum(g.n * (4 * g.m + 22 * g.n) for g in gs)) + 12.0 * arcs
    achieved = alg / (ms / 1e3) / 1e9
    t0 = time.perf_counter()
    done_w, k = 0.0, 0
    while time.perf_counter() - t0 < c.cpu_seconds and k < len(gs):
        oracle.bc(gs[k], threads=os.cpu_count() or 1)
        done_w += gs[k].n * gs[k].m
        k += 1
    cdt = time.perf_counter() - t0
    return {"metric": METRIC, "unit": UNIT, "value": work / (ms / 1e3), "ms_per_step": ms,
            "config": {"workload": f"{len(gs)} graphs, n log-uniform [50,5000], ER deg 6 / BA m=3, all sources",
                       "graphs_per_s": len(gs) / (ms / 1e3), "batch": best,
                       "sum_n": int(sum(g.n for g in gs)), "sum_nm": work, "dag_arcs": arcs},
            "roofline": {"bound": "hbm", "kernel": "k_many", "achieved": achieved, "peak": c.hbm, "unit": "GB/s",
                         "frac": achieved / c.hbm, "peak_source": c.hbm_kind, "traffic": None,
                         "algorithmic_bytes": alg,
                         "note": "per source 4m + 12a + 22n bytes over one persistent launch (replay time)"},
            "error_vs_oracle": err,
            "cpu_baseline": {"value": done_w / cdt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"first {k} graphs, all sources ({cdt:.1f} s)"}}


def cfg_directed(c):
    import torch
    nat = c.native
    g = G.rmat_directed()
    src = torch.arange(g.n, dtype=torch.int32, device="cuda")
    with nat.Graph.from_csr(g, trust_input=True) as h:
        ms = c.timed(lambda: (h.run(src, batch=BATCH, stream=c.stream), h.result()))
    return {"metric": METRIC, "unit": UNIT, "value": g.n * g.m / (ms / 1e3), "ms_per_step": ms,
            "config": {"workload": f"R-MAT s16 ef16 kept directed, weakly connected LCC (n={g.n}, "
                                   f"arcs={g.m}), all sources, batch {BATCH}", "metric_m": "arcs"},
            "cpu_baseline": _oracle_rate(g, np.arange(g.n, dtype=np.int32), c.cpu_seconds)}


def cfg_wdense(c):
    nat = c.native
    g = G.gnp_weighted(4096, 0.05, 10)
    with nat.Graph.from_csr(g, trust_input=True) as h:
        ms_d = c.timed(lambda: (h.run(flags=nat.BC_DENSE, stream=c.stream), h.result()))
        h.run(flags=nat.BC_DENSE | nat.BC_TIMING, stream=c.stream)
        h.result()
        kinds = {nat.KERNEL_NAMES[k]: h.kernel_time(k) for k in nat.KERNEL_NAMES}
        ms_s = c.timed(lambda: (h.run(stream=c.stream), h.result()), 2, 1)
    steps, mp_ms = kinds["dense"]
    # one product step: 512 sources x n x n (add + min) pairs; lanes x clock = 1 issue per lane
    elem = steps * 512.0 * g.n * g.n
    lane_peak = 152 * 128 * 2.07e9
    ach = elem / (mp_ms / 1e3)
    return {"metric": METRIC, "unit": UNIT, "value": g.n * g.m / (ms_d / 1e3), "ms_per_step": ms_d,
            "config": {"workload": f"G(n=4096, p=0.05) weighted U{{1..10}} (m={g.m}), all sources, "
                                   "BC_DENSE: distance products with counts + pair formula",
                       "kernels_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in kinds.items()},
                       "product_steps": steps},
            "roofline": {"bound": "alu", "kernel": "k_mp_step", "achieved": ach / 1e12, "peak": lane_peak / 1e12,
                         "unit": "T (min,+) elements/s", "frac": ach / lane_peak,
                         "peak_source": "152 SMs x 128 int32 lanes x 2.07 GHz, one element per lane-instruction",
                         "traffic": None},
            "vs_bucket_kernel_same_graph": {"ms": ms_s, "value": g.n * g.m / (ms_s / 1e3)},
            "cpu_baseline": _oracle_rate(g, np.arange(g.n, dtype=np.int32), c.cpu_seconds)}


def cfg_pairs(c):
    nat = c.native
    g = G.gnp(4096, 0.01)
    with nat.Graph.from_csr(g, trust_input=True) as h:
        ms_p = c.timed(lambda: (h.run(flags=nat.BC_PAIRS, stream=c.stream), h.result()))
        h.run(flags=nat.BC_PAIRS | nat.BC_TIMING, stream=c.stream)
        h.result()
        kinds = {nat.KERNEL_NAMES[k]: h.kernel_time(k) for k in nat.KERNEL_NAMES}
        ms_s = c.timed(lambda: (h.run(stream=c.stream), h.result()), 2, 1)
    _, pair_ms = kinds["backward"]
    triples = float(g.n) ** 3
    lane_peak = 152 * 128 * 2.07e9
    ach = triples / (pair_ms / 1e3)
    return {"metric": METRIC, "unit": UNIT, "value": g.n * g.m / (ms_p / 1e3), "ms_per_step": ms_p,
            "config": {"workload": f"G(n=4096, p=0.01) (m={g.m}), all pairs, BC_PAIRS: forward rows + "
                                   "Algorithm 2 pair formula",
                       "kernels_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in kinds.items()}},
            "roofline": {"bound": "alu", "kernel": "k_pair_bc (+ prep, reduce)", "achieved": ach / 1e12,
                         "peak": lane_peak / 1e12, "unit": "T (s,v,t) triples/s", "frac": ach / lane_peak,
                         "peak_source": "152 SMs x 128 lanes x 2.07 GHz, one triple per lane-instruction",
                         "traffic": None},
            "vs_level_sweep_same_graph": {"ms": ms_s, "value": g.n * g.m / (ms_s / 1e3)},
            "cpu_baseline": _oracle_rate(g, np.arange(g.n, dtype=np.int32), c.cpu_seconds)}


CONFIGS = {"er1024": cfg_er1024, "grid": cfg_grid, "gnp": cfg_gnp, "many": cfg_many,
           "directed": cfg_directed, "wdense": cfg_wdense, "pairs": cfg_pairs}
# the workloads measured beside the R-MAT line by default (ER n=1024, the
# weighted grid, G(8192, 0.05), the 2000-graph set); the others on request
# with --workload
DEFAULT_EXTRA = ("er1024", "grid", "gnp", "many")


def run_extra(args):
    """One other configuration as its own JSON line (not the default line)."""
    c = Ctx(args, args.cpu_seconds)
    fn = CONFIGS[args.workload]
    line = fn(c, full=True) if args.workload == "gnp" else fn(c)
    line.update(n_gpus=1, steps=args.steps, warmup=args.warmup, higher_is_better=True, data="synthetic",
                workload=args.workload)
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Profiling mode: one run of one workload's hot path on its first
    --sources sources (default one batch of 256 on one lane: a small case for
    ncu), nothing else."""
    import torch
    from paper_0809_1906_gb300 import native
    native.load()
    wl = args.workload
    flags = 0
    if wl == "rmat":
        g, desc = workload()
    elif wl == "er1024":
        g, desc = G.er_hamiltonian(), "er1024"
    elif wl == "grid":
        g, desc = G.grid_longrange(), "grid512 weighted"
    elif wl == "gnp":
        g, desc, flags = G.gnp(8192, 0.05), "gnp8192 dense", native.BC_DENSE
    else:
        # a capture-sized set: the per-CTA workspaces grow with the largest n
        gs = G.many_graphs(args.sources or 200, 50, args.nmax)
        hs = [native.Graph.from_csr(x, trust_input=True) for x in gs]
        with native.ManyPlan(hs, batch=256) as plan:
            plan.run()
            code, _, rerun = plan.result()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": "many", "graphs": len(gs), "status": code}), flush=True)
        return
    k = min(args.sources or 256, g.n)
    if wl == "grid":
        src = G.sample_sources(g.n, k, 33)
    elif wl == "rmat" and k < g.n:
        src = G.sample_sources(g.n, k, 34)  # a representative batch, not the hub-heavy first one
    else:
        src = np.arange(k, dtype=np.int32)
    with native.Graph.from_csr(g, trust_input=True) as hp:
        hp.run(src, batch=args.batch if wl == "rmat" else 0, flags=flags)
        out, code, _ = hp.result()
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": desc, "sources": k, "status": code, "bc_sum": float(out.sum())}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--extra-cpu-seconds", type=float, default=4.0,
                    help="oracle time budget of each extra configuration's cpu_baseline")
    ap.add_argument("--plain-sources", type=int, default=1024)
    ap.add_argument("--err-sources", type=int, default=1024,
                    help="sources of the R-MAT sample compared with the FP64 oracle")
    ap.add_argument("--profile", action="store_true",
                    help="profiling mode: one bc_run over the first --sources sources (default 256), nothing else")
    ap.add_argument("--sources", type=int, default=0)
    ap.add_argument("--nmax", type=int, default=1000, help="--profile --workload many: largest graph")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--workload", default="rmat", choices=["rmat"] + sorted(CONFIGS),
                    help="rmat (default, the reported line) or one of the other configurations alone")
    ap.add_argument("--extra", default=",".join(DEFAULT_EXTRA),
                    help="configurations measured beside the R-MAT line (comma list, or 'none')")
    ap.add_argument("--write-traffic", metavar="CSV", default=None,
                    help="write profiles/traffic_rmat.json from an ncu CSV capture of --profile, then exit")
    ap.add_argument("--traffic-command", default="", help="the ncu command line recorded with --write-traffic")
    ap.add_argument("--write-traffic-grid", metavar="CSV", default=None,
                    help="write profiles/traffic_grid.json from an ncu CSV capture of --profile --workload grid "
                         "over --sources sources, then exit")
    args = ap.parse_args()
    if args.write_traffic:
        return write_traffic(args.write_traffic, args.traffic_command)
    if args.write_traffic_grid:
        if args.sources <= 0:
            ap.error("--write-traffic-grid needs --sources: the sources the captured launches covered")
        return write_traffic_grid(args.write_traffic_grid, args.sources, args.traffic_command)
    args.warmup = max(args.warmup, 3)
    if args.profile:
        return run_profile(args)
    if args.workload != "rmat" and args.impl == "ours":
        return run_extra(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_0809_1906_gb300 import native
    from paper_0809_1906_gb300.sharding import shard_sources, reduce_partials_device
    native.load()
    g, desc = workload()
    n, m = g.n, g.m
    # one all-sources job split over the ranks: disjoint strided batches of
    # 256 sources per rank, then one rank-ordered sum of the n FP64 partial
    # vectors (no collective inside the sweep)
    src = shard_sources(np.arange(n, dtype=np.int32), rank, world, BATCH)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    h = native.Graph.from_csr(g, trust_input=True)
    src_d = torch.from_numpy(src).cuda()
    out_d = torch.empty(n, dtype=torch.float64, device="cuda")

    def step(flags):
        h.run(src_d, batch=BATCH, flags=flags, stream=stream)
        h.result(out_d)
        return reduce_partials_device(out_d) if dist else out_d

    for _ in range(args.warmup):
        step(0)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM, L2 flushed between steps
    times, launches = [], 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(0)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            launches += h.launch_count()
    torch.cuda.synchronize()
    total_ms = sum(times)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n * m / (ms_per_step / 1000.0)  # the whole job: every source of the graph once
    arcs, depth_sum = h.run_stats()

    # ---- per-launch CUDA events of every kernel (same steps, BC_TIMING)
    ktime = {}
    for _ in range(2):
        flush.fill_(1.0)
        step(native.BC_TIMING)
        for kind, name in native.KERNEL_NAMES.items():
            cnt, tot = h.kernel_time(kind)
            ktime[name] = (cnt, tot)
    fwd_b, bwd_b = algorithmic_bytes(n, m, arcs, src.size, BATCH)
    peak, peak_kind = peaks()
    f_ms = ktime["forward"][1]
    b_ms = ktime["backward"][1]
    dom, dom_bytes, dom_ms, dom_cnt = ("backward", bwd_b, b_ms, ktime["backward"][0]) if b_ms >= f_ms else \
        ("forward", fwd_b, f_ms, ktime["forward"][0])
    achieved = dom_bytes / (dom_ms / 1000.0) / 1e9
    traffic = measured_traffic(dom)
    other = "forward" if dom == "backward" else "backward"
    o_b, o_ms = (fwd_b, f_ms) if other == "forward" else (bwd_b, b_ms)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    src_h = torch.from_numpy(src).pin_memory()
    out_h = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    if dist:
        dist.barrier()
    for i in range(1 + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        he = native.Graph(n, rp_h, col_h, trust_input=True)
        he.run(src_h, batch=BATCH, stream=stream)
        if dist:
            he.result(out_d)
            out_h.copy_(reduce_partials_device(out_d))
        else:
            he.result(out_h)
        he.close()
        dt = (time.perf_counter() - t0) * 1000.0
        if i > 0:
            e2e_ms.append(dt)
    e2e_step = statistics.median(e2e_ms)
    if dist:
        t = torch.tensor([e2e_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step = float(t.item())
    e2e_value = n * m / (e2e_step / 1000.0)
    h2d = (g.row_ptr.nbytes + g.col.nbytes + src.nbytes)
    d2h = n * 8 + 4

    line = None
    if rank == 0:
        import oracle
        # ---- plain one-source-per-launch GPU Brandes on a bounded sample
        plain_k = min(args.plain_sources, n)
        psrc = torch.from_numpy(np.arange(plain_k, dtype=np.int32)).cuda()
        h.run(psrc, flags=native.BC_PLAIN, stream=stream)
        h.result(out_d)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.run(psrc, flags=native.BC_PLAIN, stream=stream)
        h.result(out_d)
        b.record(stream)
        b.synchronize()
        plain_value = plain_k * m / (a.elapsed_time(b) / 1000.0)
        # ---- error against the FP64 oracle on a bounded seeded sample of sources
        esrc = G.sample_sources(n, min(args.err_sources, n), 902)
        h.run(esrc, batch=BATCH, stream=stream)
        got, _, _ = h.result()
        err = err_stats(got, oracle.bc(g, esrc)["bc"], n, f"{esrc.size} seeded sources, batch {BATCH}")
        cpu_v, cores, k, dt = cpu_oracle_rate(g, args.cpu_seconds)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u64+f32 (BC f64)", "data": "synthetic",
            "config": {"workload": desc, "n": n, "m": m, "sources": n, "batch": BATCH},
            "config_detail": {"sources_rank0": int(src.size),
                              "parallelism": f"sources sharded over {world} rank(s) in strided batches, one FP64 sum",
                              "l2": "flushed (512 MB write) between timed steps",
                              "dag_arcs_per_source": arcs / max(src.size, 1), "depth_sum": depth_sum},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": traffic, "algorithmic_bytes_per_launch": dom_bytes / max(dom_cnt, 1),
                         "avg_launch_ms": dom_ms / max(dom_cnt, 1), "launches": dom_cnt,
                         "kernel_timing": "BC_TIMING pass: one lane, CUDA events around every launch",
                         f"{other}_frac": o_b / (o_ms / 1000.0) / 1e9 / peak,
                         "step_achieved": (fwd_b + bwd_b) / (ms_per_step / 1000.0) / 1e9,
                         "step_frac": (fwd_b + bwd_b) / (ms_per_step / 1000.0) / 1e9 / peak,
                         "step_note": "forward + backward algorithmic bytes / ms_per_step (concurrent lanes)"},
            "kernels_ms": {k2: {"launches": v[0], "total_ms": v[1]} for k2, v in ktime.items()},
            "error_vs_oracle": err,
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{k} seeded sources of the same graph ({dt:.1f} s, OpenMP over sources)"},
            "vs_plain_gpu": {"value": plain_value, "unit": UNIT, "speedup": value / plain_value,
                             "sample": f"first {plain_k} sources, one source per launch sequence"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_step},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
    h.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        # the other configurations, each with its own roofline, oracle error
        # and cpu_baseline (rank 0 only, after the timed R-MAT region)
        extra = [x for x in args.extra.split(",") if x and x != "none"]
        if extra:
            c = Ctx(args, args.extra_cpu_seconds)
            line["configs"] = {}
            for name in extra:
                try:
                    line["configs"][name] = CONFIGS[name](c)
                except Exception as e:  # a failing extra configuration must not hide the main line
                    line["configs"][name] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
