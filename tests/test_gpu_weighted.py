"""GPU parity of the weighted path (integer buckets, tie-aware sigma) against
the oracle's binary-heap Dijkstra Brandes."""
import math

import numpy as np
import pytest

import oracle
from paper_0809_1906_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_0809_1906_gb300 import native
    native.load()
    return native


def assert_bc_close(got, ref, n, what=""):
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * max(n, 1))
    err = np.abs(got - ref)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"{what}: {bad.size} off, worst {err.max():.3e} (rel {np.max(err / np.maximum(np.abs(ref), 1e-30)):.2e})"
    return float(np.max(err / np.maximum(np.abs(ref), 1.0)))


def check(nat, g, sources=None, batch=0, rows=8, flags=0):
    """The default run (an undirected graph runs on its relabelled copy) or,
    with BC_KEEP_ORDER, the caller's numbering: against the oracle."""
    ref = oracle.bc(g, sources)
    with nat.Graph.from_csr(g) as h:
        h.run(sources, batch=batch, flags=flags)
        got, code, _ = h.result()
        ns = g.n if sources is None else len(sources)
        hs = h.source_hashes(ns)
        assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]), g.name
        assert np.array_equal(hs["hash_dist"], ref["hash_dist"]), g.name
        assert np.array_equal(hs["reach"], ref["reach"]), g.name
        assert code == (nat.BC_WARN_SIGMA_OVERFLOW if ref["flags"] & 1 else nat.BC_OK)
        rel = assert_bc_close(got, ref["bc"], g.n, g.name)
        if rows:
            src = np.arange(g.n, dtype=np.int32) if sources is None else np.asarray(sources, np.int32)
            pick = src[:rows]
            sig, dist, _ = h.forward_rows(pick, flags=flags)
            for i, s in enumerate(pick.tolist()):
                o = oracle.source(g, s, with_delta=False)
                assert np.array_equal(dist[i], o["dist"].astype(np.int32)), (g.name, s)
                assert np.array_equal(sig[i], o["sigma"]), (g.name, s)
    return rel


@pytest.mark.parametrize("seed", range(8))
def test_small_weighted_ties(nat, seed):
    n = [9, 20, 50, 120, 333, 600, 1000, 64][seed]
    g = G.random_small(n, min(0.5, 4.0 / n), 1200 + seed, wmax=3, connect=seed % 3 != 0)
    check(nat, g, batch=[0, 1, 7, 64][seed % 4])


@pytest.mark.parametrize("seed", range(4))
def test_caller_numbering_matches_oracle(nat, seed):
    """BC_KEEP_ORDER keeps the caller's vertex ids on the weighted sweep."""
    n = [50, 333, 1000, 64][seed]
    g = G.random_small(n, min(0.5, 4.0 / n), 1300 + seed, wmax=3, connect=seed % 2 == 0)
    check(nat, g, batch=[0, 7][seed % 2], flags=nat.BC_KEEP_ORDER)


def test_relabelled_and_caller_numbering_agree(nat):
    """Both numberings give the same rows and summaries bit for bit; BC only
    differs by summation order."""
    big = G.grid_longrange(side=96, frac=0.05, wmax=100, seed=77)
    src = G.sample_sources(big.n, 300, 5)
    with nat.Graph.from_csr(big) as h:
        out = {}
        for fl in (0, nat.BC_KEEP_ORDER):
            h.run(src, flags=fl)
            bc, code, _ = h.result()
            hs = h.source_hashes(len(src))
            sig, dist, _ = h.forward_rows(src[:16], flags=fl)
            out[fl] = (bc, hs, sig, dist)
        a, b = out[0], out[nat.BC_KEEP_ORDER]
        for k in ("hash_sigma", "hash_dist", "reach"):
            assert np.array_equal(a[1][k], b[1][k]), k
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
        assert_bc_close(a[0], b[0], big.n, "relabelled vs caller numbering")
    ref = oracle.bc(big, src)
    assert_bc_close(a[0], ref["bc"], big.n, "relabelled vs oracle")


def test_uniform_weight_equals_unweighted(nat):
    g1 = G.grid_graph(20)
    g5 = G.grid_graph(20, w=5)
    with nat.Graph.from_csr(g1) as h1, nat.Graph.from_csr(g5) as h5:
        h1.run()
        h5.run()
        a, _, _ = h1.result()
        b, _, _ = h5.result()
    assert np.allclose(a, b, rtol=2e-5)


def test_subgrid64_all_sources(nat):
    """Induced 64x64 block of the 512x512 long-range grid, every source."""
    g = G.induced_subgrid(G.grid_longrange(), 512, 64)
    rel = check(nat, g)
    print(f"subgrid64 max rel err {rel:.2e}")


def test_grid512_sampled_sources(nat):
    """Full 512x512 grid + 5% long-range edges, w ~ U{1..100}: the launch
    configuration of the full run on 4096 sampled sources, checked on
    per-source hashes of a sample, BC over 48 sources, and the identity
    sum_v delta = sum_t ... via reach."""
    g = G.grid_longrange()
    src = G.sample_sources(g.n, 4096, 33)
    with nat.Graph.from_csr(g) as h:
        h.run(src)
        got, code, _ = h.result()
        hs = h.source_hashes(src.size)
        assert code == nat.BC_OK
        pick = np.arange(0, 4096, 256)
        ref = oracle.bc(g, src[pick])
        assert np.array_equal(hs["hash_sigma"][pick], ref["hash_sigma"])
        assert np.array_equal(hs["hash_dist"][pick], ref["hash_dist"])
        assert np.all(hs["reach"] == g.n)
        sub = src[:48]
        h.run(sub)
        got, _, _ = h.result()
        rel = assert_bc_close(got, oracle.bc(g, sub)["bc"], g.n, "grid512 48 sources")
        print(f"grid512 max rel err {rel:.2e}")


def test_weighted_overflow_flag(nat):
    g = G.grid_graph(35, w=2)
    with nat.Graph.from_csr(g) as h:
        sig, dist, code = h.forward_rows(np.array([0], np.int32))
    assert code == nat.BC_WARN_SIGMA_OVERFLOW
    assert int(sig[0, -1]) == math.comb(68, 34) % (1 << 64) and dist[0, -1] == 136


def test_weight_limit(nat):
    g = G.path_graph(3)
    big = G.csr_from_edges(3, [0, 1], [1, 2], [5000, 1])
    with nat.Graph.from_csr(big) as h:
        with pytest.raises(nat.BcError) as e:
            h.run()
        assert e.value.code == nat.BC_ERR_UNSUPPORTED
    with pytest.raises(nat.BcError) as e:
        nat.Graph(3, g.row_ptr, g.col, np.array([1, 0, 0, 1], np.int32))
    assert e.value.code == nat.BC_ERR_WEIGHT


def test_counts_beyond_32_bits_fall_back_exactly(nat):
    """Unit weights on a 20 x 20 grid given as a weighted graph: counts up to
    C(38,19) > 2^32 exceed the packed kernel's 32-bit sigma, so those sources
    are recomputed with 64-bit counts; sources whose counts stay small (a
    ragged wave mixing both kinds) keep the packed result. Rows, summaries and
    BC match the oracle."""
    g0 = G.grid_graph(20)
    g = G.Graph(g0.n, g0.row_ptr, g0.col, np.ones_like(g0.col), "grid20w")
    src = np.array([0, 210, 399, 19, 55, 380, 7, 200], np.int32)
    check(nat, g, sources=src, batch=5)


def test_packed_and_64bit_overflow_flag(nat):
    """35 x 35 unit-weight grid: sigma(corner, far corner) = C(68,34) >= 2^64;
    the fallback keeps the low 64 bits and raises the overflow warning."""
    g0 = G.grid_graph(35)
    g = G.Graph(g0.n, g0.row_ptr, g0.col, np.ones_like(g0.col), "grid35w")
    with nat.Graph.from_csr(g) as h:
        sig, dist, code = h.forward_rows(np.array([0, 17], np.int32))
    assert code == nat.BC_WARN_SIGMA_OVERFLOW
    assert int(sig[0, -1]) == math.comb(68, 34) % (1 << 64) and dist[0, -1] == 68
    o = oracle.source(g, 17, with_delta=False)
    assert np.array_equal(sig[1], o["sigma"]) and np.array_equal(dist[1], o["dist"].astype(np.int32))



def test_waves_on_two_lanes_with_deferred_redo(nat):
    """Waves of 3 sources alternate between two lanes; sources whose counts
    pass 2^32 (unit-weight 20 x 20 grid, far corners) are recomputed after
    the last wave. BC, summaries and the forward rows of every source match
    the oracle, and two runs give identical BC."""
    g0 = G.grid_graph(20)
    g = G.Graph(g0.n, g0.row_ptr, g0.col, np.ones_like(g0.col), "grid20w")
    src = np.array([0, 210, 399, 19, 55, 380, 7, 200, 20, 389, 150, 3, 396], np.int32)
    check(nat, g, sources=src, batch=3, rows=0)
    with nat.Graph.from_csr(g) as h:
        sig, dist, code = h.forward_rows(src, batch=3)
        h.run(src, batch=3)
        a, _, _ = h.result()
        h.run(src, batch=3)
        b, _, _ = h.result()
    assert np.array_equal(a, b)
    for i, s in enumerate(src.tolist()):
        o = oracle.source(g, s, with_delta=False)
        assert np.array_equal(dist[i], o["dist"].astype(np.int32)), s
        assert np.array_equal(sig[i], o["sigma"]), s
