"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

sigma and distances must match bit for bit (full rows, and the per-source
summary hashes of every source); BC must be within
max(1e-5 * |ref|, 1e-6 * n) of the FP64 oracle (dependencies run in FP32 on
the device, the sum over sources in FP64)."""
import math

import numpy as np
import pytest

import oracle
from paper_0809_1906_gb300 import graphs as G

pytestmark = pytest.mark.gpu

REL, ABS_PER_N = 1e-5, 1e-6


@pytest.fixture(scope="module")
def nat():
    from paper_0809_1906_gb300 import native
    native.load()
    return native


def assert_bc_close(got, ref, n, what=""):
    tol = np.maximum(REL * np.abs(ref), ABS_PER_N * max(n, 1))
    err = np.abs(got - ref)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"{what}: {bad.size} vertices off, worst {err.max():.3e} at {int(np.argmax(err))}"


def check_graph(nat, g, sources=None, batch=0, flags=0, chunk=0, rows=True):
    ref = oracle.bc(g, sources)
    with nat.Graph.from_csr(g) as h:
        h.run(sources, batch=batch, flags=flags, chunk=chunk)
        got, code, st = h.result()
        ns = g.n if sources is None else len(sources)
        hs = h.source_hashes(ns)
        assert_bc_close(got, ref["bc"], g.n, g.name)
        assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]), g.name
        assert np.array_equal(hs["hash_dist"], ref["hash_dist"]), g.name
        assert np.array_equal(hs["dist_sum"], ref["dist_sum"]), g.name
        assert np.array_equal(hs["reach"], ref["reach"]), g.name
        assert code == (nat.BC_WARN_SIGMA_OVERFLOW if ref["flags"] & 1 else nat.BC_OK)
        # the shortest-path DAG arcs the device counted (the roofline's a)
        arcs, _ = h.run_stats()
        assert arcs == int(ref["arcs"].sum()), (g.name, arcs, int(ref["arcs"].sum()))
        if rows and not (flags & nat.BC_PLAIN):
            src = np.arange(g.n, dtype=np.int32) if sources is None else np.asarray(sources, np.int32)
            pick = src[: min(len(src), 40)]
            sig, dist, _ = h.forward_rows(pick, batch=batch)
            for i, s in enumerate(pick.tolist()):
                o = oracle.source(g, s, with_delta=False)
                assert np.array_equal(dist[i], o["dist"].astype(np.int32)), (g.name, s)
                assert np.array_equal(sig[i], o["sigma"]), (g.name, s)
    return got


SMALL = [G.path_graph(2), G.path_graph(9), G.path_graph(40), G.cycle_graph(9), G.cycle_graph(13),
         G.star_graph(30), G.complete_graph(12), G.complete_bipartite(3, 5), G.grid_graph(8),
         G.layered_biclique(5, 7)]


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
@pytest.mark.parametrize("batch", [32, 256])
def test_closed_form_graphs(nat, g, batch):
    check_graph(nat, g, batch=batch)


@pytest.mark.parametrize("batch", [32, 64, 128, 256])
@pytest.mark.parametrize("chunk", [0, 4])
def test_er1024_all_sources(nat, batch, chunk):
    """n=1024 G(n, 4096) + Hamiltonian path, every source; chunk=4 splits
    every vertex of degree > 4 so the partial-combine path runs everywhere."""
    g = G.er_hamiltonian()
    check_graph(nat, g, batch=batch, chunk=chunk)


def test_plain_path_matches(nat):
    g = G.er_hamiltonian(300, 1200, 11)
    check_graph(nat, g, flags=nat.BC_PLAIN)
    check_graph(nat, G.star_graph(17), flags=nat.BC_PLAIN)


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_ragged_batches(nat, seed):
    """Disconnected random graphs, source counts that leave a ragged last batch."""
    n = [50, 77, 130, 301, 513, 1000][seed]
    g = G.random_small(n, 2.5 / n, 900 + seed, connect=seed % 2 == 0)
    src = G.sample_sources(n, n - 7 if n > 40 else n, 5 + seed)
    check_graph(nat, g, sources=src, batch=64, chunk=8)


def test_duplicate_and_single_sources(nat):
    g = G.er_hamiltonian(200, 700, 3)
    check_graph(nat, g, sources=np.array([5, 5, 9, 5], np.int32))
    check_graph(nat, g, sources=np.array([199], np.int32))


def test_empty_and_trivial(nat):
    g1 = G.csr_from_edges(1, [], [])
    with nat.Graph.from_csr(g1) as h:
        h.run()
        out, code, _ = h.result()
        assert out.tolist() == [0.0] and code == 0
    g = G.path_graph(5)
    with nat.Graph.from_csr(g) as h:
        h.run(np.zeros(0, np.int32))
        out, code, _ = h.result()
        assert np.all(out == 0)
    iso = G.csr_from_edges(6, [0, 1], [1, 2])  # vertices 3..5 isolated
    check_graph(nat, iso)


def test_halve_and_accumulate(nat):
    g = G.path_graph(17)
    with nat.Graph.from_csr(g) as h:
        h.run(flags=nat.BC_HALVE)
        half, _, _ = h.result()
        i = np.arange(1, 18)
        assert np.allclose(half, (i - 1) * (17 - i), rtol=1e-6)
        h.run(np.arange(0, 8, dtype=np.int32))
        h.run(np.arange(8, 17, dtype=np.int32), flags=nat.BC_ACCUMULATE)
        acc, _, _ = h.result()
        assert np.allclose(acc, 2 * (i - 1) * (17 - i), rtol=1e-6)


def test_sigma_overflow_flag_grid35(nat):
    """35x35 grid: sigma(corner, far corner) = C(68,34) >= 2^64 -> warning;
    the low 64 bits still match (sums wrap mod 2^64 on both sides)."""
    g = G.grid_graph(35)
    with nat.Graph.from_csr(g) as h:
        sig, dist, code = h.forward_rows(np.array([0], np.int32))
        assert code == nat.BC_WARN_SIGMA_OVERFLOW
        assert int(sig[0, -1]) == math.comb(68, 34) % (1 << 64)
        h.run(np.array([0, 1], np.int32))
        _, code, st = h.result()
        assert code == nat.BC_WARN_SIGMA_OVERFLOW and st & nat.BC_STATUS_SIGMA_OVERFLOW
    g34 = G.grid_graph(34)
    with nat.Graph.from_csr(g34) as h:
        sig, _, code = h.forward_rows(np.array([0], np.int32))
        assert code == nat.BC_OK and int(sig[0, -1]) == math.comb(66, 33)


def test_layered_biclique_carries(nat):
    g = G.layered_biclique(17, 16)
    o = oracle.source(g, 0, with_delta=False)
    with nat.Graph.from_csr(g) as h:
        sig, dist, code = h.forward_rows(np.array([0], np.int32))
    assert np.array_equal(sig[0], o["sigma"]) and code == nat.BC_WARN_SIGMA_OVERFLOW


def test_deterministic(nat):
    g = G.er_hamiltonian(2000, 9000, 8)
    with nat.Graph.from_csr(g) as h:
        h.run(batch=128, chunk=16)
        a, _, _ = h.result()
        h.run(batch=128, chunk=16)
        b, _, _ = h.result()
    assert np.array_equal(a, b)


def test_landmark_order_matches_given_order(nat):
    """Batches formed in landmark order (the default) and in the given order
    give the same per-source summaries, both in the caller's order, and BC
    within tolerance of the oracle; the source list is shuffled, holds
    duplicates and leaves a ragged last batch."""
    g = G.er_hamiltonian(2000, 9000, 8)
    rng = np.random.default_rng(3)
    src = rng.integers(0, g.n, 700).astype(np.int32)
    ref = oracle.bc(g, src)
    with nat.Graph.from_csr(g) as h:
        h.run(src, batch=64)
        a, _, _ = h.result()
        ha = h.source_hashes(len(src))
        h.run(src, batch=64, flags=nat.BC_KEEP_ORDER)
        b, _, _ = h.result()
        hb = h.source_hashes(len(src))
    for k in ("hash_sigma", "hash_dist", "dist_sum", "reach"):
        assert np.array_equal(ha[k], ref[k]), k
        assert np.array_equal(hb[k], ref[k]), k
    assert_bc_close(a, ref["bc"], g.n, "landmark order")
    assert_bc_close(b, ref["bc"], g.n, "given order")


def test_device_pointer_inputs(nat):
    import torch
    g = G.er_hamiltonian(500, 2000, 4)
    ref = oracle.bc(g)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    src = torch.arange(g.n, dtype=torch.int32, device="cuda")
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    h = nat.Graph(g.n, rp, col)
    try:
        h.run(src, stream=torch.cuda.current_stream())
        h.result(out)
    finally:
        h.close()
    assert_bc_close(out.cpu().numpy(), ref["bc"], g.n)


def test_rejects_bad_input(nat):
    with pytest.raises(nat.BcError) as e:
        nat.Graph(3, np.array([0, 1, 1, 1], np.int32), np.array([1], np.int32))  # missing reverse arc
    assert e.value.code == nat.BC_ERR_NOT_SYMMETRIC
    g = G.path_graph(4)
    with nat.Graph.from_csr(g) as h:
        with pytest.raises(nat.BcError) as e:
            h.run(np.array([4], np.int32))
        assert e.value.code == nat.BC_ERR_ARG
        with pytest.raises(nat.BcError):
            h.run(batch=48)


@pytest.mark.slow
def test_rmat_full_size_bench_configuration(nat):
    """The R-MAT scale-16 LCC at full size, every source, batch 256: the
    benchmark's launch configuration (eight concurrent lanes, landmark-ordered
    batches). BC of all 46,894 sources element by element against the FP64
    oracle over the same sources (all host cores), every source's sigma and
    distance summaries bit for bit, the device's DAG-arc count against the
    oracle's, and the identity sum_v BC(v) = sum_s (sum_t d(s,t) - (reach_s - 1))."""
    g = G.rmat_lcc()
    ref = oracle.bc(g)
    with nat.Graph.from_csr(g) as h:
        h.run(batch=256)
        bc, code, _ = h.result()
        hs = h.source_hashes(g.n)
        arcs, _ = h.run_stats()
    assert code == nat.BC_OK
    assert_bc_close(bc, ref["bc"], g.n, "rmat all sources")
    for k in ("hash_sigma", "hash_dist", "dist_sum", "reach"):
        assert np.array_equal(hs[k], ref[k]), k
    assert arcs == int(ref["arcs"].sum())
    rhs = float((hs["dist_sum"] - (hs["reach"] - 1)).sum())
    assert abs(bc.sum() - rhs) <= 1e-6 * rhs
    nz = ref["bc"] > 0
    rel = float(np.max(np.abs(bc[nz] - ref["bc"][nz]) / ref["bc"][nz]))
    print(f"rmat all sources: max relative error {rel:.3e} against the FP64 oracle")


def test_autotuner_choice_runs_correctly(nat, tmp_path, monkeypatch):
    """The library's tuner picks launch options and installs them as the
    handle's default: bc_run with NULL options then runs with that choice
    (bc_last_options), correctly; a second process-level call is served from
    the JSON cache and installs the same choice on a fresh handle."""
    from paper_0809_1906_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    g = G.er_hamiltonian(3000, 15000, 9)
    ref = oracle.bc(g)
    with nat.Graph.from_csr(g) as h:
        choice = autotune.tune_graph(g, h, sample=512)
        assert choice["batch"] in (64, 128, 256) and choice["chunk"] in (128, 256, 512) and not choice["cached"]
        assert choice["beta"] in (0.0, pytest.approx(1 / 256), pytest.approx(1 / 16))  # 0: the default 1/64
        h.run(default_options=True)
        got, code, _ = h.result()
        used = h.last_options()
        assert (used.batch, used.chunk) == (choice["batch"], choice["chunk"])
        assert_bc_close(got, ref["bc"], g.n, "tuned defaults")
        hs = h.source_hashes(g.n)
        assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"])
        h.set_default_options(None)  # back to the built-in defaults
        h.run(default_options=True)
        assert h.last_options().batch == 0
    assert (tmp_path / "tune.json").exists()
    with nat.Graph.from_csr(g) as h2:
        again = autotune.tune_graph(g, h2)
        assert again["cached"] and again["batch"] == choice["batch"]
        h2.run(default_options=True)
        assert h2.last_options().chunk == choice["chunk"]


@pytest.mark.parametrize("batch", [32, 64])
def test_concurrent_lanes_deep_batches(nat, batch):
    """Many batches run on concurrent lanes; a path of 300 vertices is deeper
    than the starting level capacity, so the capacity grows (every lane's
    unfinished batch starts over) several times within one run."""
    for g in (G.path_graph(300), G.random_small(700, 0.004, 4242, connect=True)):
        ref = oracle.bc(g)
        with nat.Graph.from_csr(g) as h:
            h.run(batch=batch)
            got, code, _ = h.result()
            hs = h.source_hashes(g.n)
            h.run(batch=batch)
            again, _, _ = h.result()
        assert code == nat.BC_OK
        tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
        assert np.all(np.abs(got - ref["bc"]) <= tol), g.name
        assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]) and np.array_equal(hs["hash_dist"], ref["hash_dist"])
        assert np.array_equal(got, again), g.name


def test_lanes_reused_across_graphs(nat):
    """Lanes of a destroyed graph serve the next graph (grown when it is
    larger, with fresh progress blocks): each result still matches."""
    for g in (G.random_small(300, 0.02, 51, connect=True), G.er_hamiltonian(1500, 6000, 52),
              G.random_small(400, 0.01, 53, connect=True), G.path_graph(200)):
        ref = oracle.bc(g)
        with nat.Graph.from_csr(g) as h:
            h.run(batch=32)
            got, code, _ = h.result()
            hs = h.source_hashes(g.n)
        assert code == nat.BC_OK
        tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
        assert np.all(np.abs(got - ref["bc"]) <= tol), g.name
        assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]), g.name


def test_parity_row_buffers_on_a_large_graph(nat):
    """n = 100,000 at 256 sources per batch: one masked-row buffer per level
    would take more than the budget, so the sweep keeps two buffers by level
    parity and the backward reads the uint64 sigma. Two batches (two lanes)
    of seeded sources against the oracle, summaries included."""
    g = G.er_hamiltonian(100_000, 400_000, 4343)
    src = G.sample_sources(g.n, 512, 44)
    ref = oracle.bc(g, src)
    with nat.Graph.from_csr(g, trust_input=True) as h:
        h.run(src, batch=256)
        got, code, _ = h.result()
        hs = h.source_hashes(src.size)
    assert code == nat.BC_OK
    tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
    assert np.all(np.abs(got - ref["bc"]) <= tol)
    assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]) and np.array_equal(hs["hash_dist"], ref["hash_dist"])


def test_sharded_run_single_rank_matches_oracle(nat):
    """The multi-GPU entry (one shard per rank, then the rank-ordered sum) on
    a world of one rank: the shard is every source."""
    from paper_0809_1906_gb300.sharding import run_sharded_gpu
    g = G.er_hamiltonian(1500, 6000, 71)
    got = run_sharded_gpu(g, batch=128)
    assert_bc_close(got, oracle.bc(g)["bc"], g.n, "sharded world 1")


def test_handles_reuse_cached_blocks(nat):
    """Destroyed handles leave their device blocks for the next ones: graphs
    of several sizes created and destroyed in turn (smaller after larger,
    which reuses larger blocks, and larger after smaller), then again after
    the cache is emptied, each against the oracle."""
    gs = [G.random_small(300, 0.02, 5, connect=True), G.random_small(120, 0.05, 6, connect=True),
          G.random_small(700, 0.006, 7, connect=True)]
    refs = [oracle.bc(g)["bc"] for g in gs]
    for rnd in range(2):
        for g, ref in zip(gs + gs[::-1], refs + refs[::-1]):
            with nat.Graph.from_csr(g) as h:
                h.run()
                got, code, _ = h.result()
            assert code == nat.BC_OK
            assert_bc_close(got, ref, g.n, f"{g.name} round {rnd}")
        nat.release_cached_memory()
