"""GPU parity for directed graphs (BC_GRAPH_DIRECTED): the forward sweep pulls
over in-arcs, the backward over out-arcs. sigma / distance summaries bit-exact
against the oracle, BC within max(1e-5 |ref|, 1e-6 n)."""
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


def check(nat, g, sources=None, rows=True, **run):
    ref = oracle.bc(g, sources)
    with nat.Graph.from_csr(g) as h:
        h.run(sources, **run)
        got, code, _ = h.result()
        ns = g.n if sources is None else len(sources)
        hs = h.source_hashes(ns)
        tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
        assert np.all(np.abs(got - ref["bc"]) <= tol), (g.name, float(np.max(np.abs(got - ref["bc"]))))
        for k in ("hash_sigma", "hash_dist", "dist_sum", "reach"):
            assert np.array_equal(hs[k], ref[k]), (g.name, k)
        assert code == (nat.BC_WARN_SIGMA_OVERFLOW if ref["flags"] & 1 else nat.BC_OK)
        if rows and not (run.get("flags", 0) & nat.BC_PLAIN):
            src = np.arange(g.n, dtype=np.int32) if sources is None else np.asarray(sources, np.int32)
            pick = src[:24]
            sig, dist, _ = h.forward_rows(pick)
            for i, s in enumerate(pick.tolist()):
                o = oracle.source(g, s, with_delta=False)
                assert np.array_equal(dist[i], o["dist"].astype(np.int32)), (g.name, s)
                assert np.array_equal(sig[i], o["sigma"]), (g.name, s)
    return got


@pytest.mark.parametrize("n", [2, 9, 40, 300])
def test_directed_path_and_cycle(nat, n):
    """One-way path BC(i) = i(n-1-i); one-way cycle (n-1)(n-2)/2 everywhere."""
    i = np.arange(n)
    got = check(nat, G.directed_path(n))
    assert np.allclose(got, i * (n - 1 - i), rtol=1e-6)
    got = check(nat, G.directed_cycle(n))
    assert np.allclose(got, np.full(n, (n - 1) * (n - 2) / 2), rtol=1e-6)


@pytest.mark.parametrize("batch", [32, 256])
@pytest.mark.parametrize("seed", range(3))
def test_directed_random_unweighted(nat, seed, batch):
    g = G.directed_random(600, 0.01 + 0.01 * seed, 1000 + seed)
    check(nat, g, batch=batch)


def test_directed_heavy_chunks_and_ragged(nat):
    """chunk=4 splits every vertex of in- or out-degree above 4 (the two sweeps
    use plans over different CSRs); a shuffled source list with duplicates."""
    g = G.directed_random(500, 0.03, 1010)
    rng = np.random.default_rng(5)
    src = rng.integers(0, g.n, 333).astype(np.int32)
    check(nat, g, sources=src, batch=64, chunk=4)
    check(nat, g, sources=src, batch=64, flags=nat.BC_KEEP_ORDER)


def test_directed_plain_path(nat):
    g = G.directed_random(300, 0.02, 1020)
    check(nat, g, flags=nat.BC_PLAIN)


@pytest.mark.parametrize("n", [1, 4, 40])
def test_kkp_tripartite_weighted(nat, n):
    """Section 2's KKP graph: BC(v_0) = n^2, every other vertex 0."""
    g = G.kkp_tripartite(n)
    got = check(nat, g)
    want = np.zeros(3 * n)
    want[n] = n * n
    assert np.allclose(got, want, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("numbering", ["relabelled", "caller"])
def test_directed_random_weighted(nat, seed, numbering):
    """The weighted sweep on its renumbered copy (out- and in-arc CSRs) and,
    with BC_KEEP_ORDER, on the caller's numbering."""
    g = G.directed_random(400, 0.02, 1030 + seed, wmax=5)
    check(nat, g, flags=nat.BC_KEEP_ORDER if numbering == "caller" else 0)


def test_directed_rejected_where_unsupported(nat):
    g = G.directed_random(100, 0.05, 1040)
    with nat.Graph.from_csr(g) as h:
        with pytest.raises(nat.BcError) as e:
            h.run(flags=nat.BC_DENSE)
        assert e.value.code == nat.BC_ERR_UNSUPPORTED
        with pytest.raises(nat.BcError) as e:
            nat.ManyPlan([h])
        assert e.value.code == nat.BC_ERR_UNSUPPORTED


def test_undirected_graph_given_as_directed(nat):
    """Both arcs of every edge given as a directed graph: same BC as the
    undirected handle."""
    g = G.er_hamiltonian(400, 1600, 12)
    src = np.repeat(np.arange(g.n), g.degrees())
    d = G.csr_from_arcs(g.n, src, g.col)
    with nat.Graph.from_csr(g) as h:
        h.run()
        a, _, _ = h.result()
    b = check(nat, d)
    assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * g.n)
