"""Pins for the CPU oracle (no GPU): enumeration, closed forms, the paper's
printed example, Algorithm 2, the algebraic forms and invariants."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_0809_1906_gb300 import graphs as G
from oracle import algebraic, brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _close(a, b, rel=1e-12, abs_=1e-12):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= abs_ + rel * np.abs(b))


def _check_against_brute(oracle_lib, g, paths=None):
    ref = brute.betweenness(g, paths)
    out = oracle_lib.bc(g)
    want = np.array([float(x) for x in ref["bc"]])
    assert _close(out["bc"], want), (g.name, out["bc"], want)
    for s in range(g.n):
        row = oracle_lib.source(g, s)
        dist = np.array([-1 if x is None else x for x in ref["dist"][s]])
        assert np.array_equal(row["dist"], dist), (g.name, s)
        lam = np.array([ref["lam"][s][v] if ref["dist"][s][v] is not None else 0 for v in range(g.n)],
                       dtype=object)
        got = np.array([int(lo) | (int(hi) << 64) for lo, hi in zip(row["sigma"], row["sigma_hi"])],
                       dtype=object)
        assert np.array_equal(got, lam), (g.name, s)
        dep = np.array([float(ref["dep"][s][v]) for v in range(g.n)])
        dep[s] = row["delta"][s]  # delta_s*(s) is not defined by Section 1.1
        assert _close(row["delta"], dep), (g.name, s)
        assert abs(row["delta"][s] - (row["reach"] - 1)) <= 1e-12 * row["reach"]  # value at the source
    return out


# ------------------------------------------------------------ enumeration

def test_pruned_enumeration_equals_raw_enumeration():
    for seed in range(6):
        g = G.random_small(6, 0.5, seed, wmax=3 if seed % 2 else 1)
        raw = brute.all_simple_paths_min(g)
        pruned = brute.shortest_paths(g)
        assert set(raw) == set(pruned)
        for k in raw:
            assert sorted(raw[k]) == sorted(pruned[k])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_every_labelled_graph_small_n(oracle_lib, n):
    """Every labelled graph on n <= 5 vertices, connected or not."""
    pairs = n * (n - 1) // 2
    for bits in range(1 << pairs):
        g = G.from_adjacency_bits(n, bits)
        _check_against_brute(oracle_lib, g)


def test_random_labelled_graphs_n6(oracle_lib):
    rs = G.Stream(6, 0)
    for bits in rs.below(300, 1 << 15).tolist():
        _check_against_brute(oracle_lib, G.from_adjacency_bits(6, int(bits)))


@pytest.mark.parametrize("seed", range(12))
def test_random_small_unweighted(oracle_lib, seed):
    n = 7 + seed % 4
    g = G.random_small(n, 0.35, 100 + seed)
    _check_against_brute(oracle_lib, g)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_weighted_ties(oracle_lib, seed):
    """Weights in {1,2,3} force ties between paths of different hop counts."""
    n = 7 + seed % 4
    g = G.random_small(n, 0.4, 200 + seed, wmax=3)
    _check_against_brute(oracle_lib, g)


def test_raw_enumeration_small_weighted(oracle_lib):
    for seed in range(4):
        g = G.random_small(7, 0.45, 300 + seed, wmax=3)
        _check_against_brute(oracle_lib, g, brute.all_simple_paths_min(g))


# ---------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 40])
def test_path_closed_form(oracle_lib, n):
    """P_n, ordered pairs: BC(v_i) = 2(i-1)(n-i), i = 1..n."""
    out = oracle_lib.bc(G.path_graph(n))["bc"]
    i = np.arange(1, n + 1)
    assert np.array_equal(out, 2.0 * (i - 1) * (n - i))


def test_paper_printed_path_values(oracle_lib):
    """Section 5's printed P_{4k+1} values (unordered = ordered / 2)."""
    with open(os.path.join(GOLDEN, "paper_path_p4k1.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for row in rows:
        k = int(row[0])
        out = oracle_lib.bc(G.path_graph(4 * k + 1))["bc"] / 2.0
        for item in row[1:]:
            pos, val = item.split(":")
            assert out[int(pos) - 1] == float(val), (k, pos)


def test_paper_cycle_erratum(oracle_lib):
    """Section 5 prints k^2 for C_{4k+1}; enumeration gives k(2k-1)."""
    with open(os.path.join(GOLDEN, "paper_cycle_c4k1.txt")) as f:
        rows = [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]
    for k, printed, true in rows:
        g = G.cycle_graph(4 * k + 1)
        out = oracle_lib.bc(g)["bc"] / 2.0
        assert np.all(out == true), (k, out)
        assert (printed == true) == (k == 1)
        if k <= 2:
            ref = brute.betweenness(g)["bc"]
            assert all(x == 2 * true for x in ref)


@pytest.mark.parametrize("n", [3, 4, 7, 30])
def test_star_closed_form(oracle_lib, n):
    out = oracle_lib.bc(G.star_graph(n))["bc"]
    assert out[0] == (n - 1) * (n - 2)
    assert np.all(out[1:] == 0)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 25])
def test_complete_graph_zero(oracle_lib, n):
    assert np.all(oracle_lib.bc(G.complete_graph(n))["bc"] == 0)


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (3, 5), (4, 4), (5, 2)])
def test_complete_bipartite(oracle_lib, a, b):
    """K_{a,b}: each A-side vertex has ordered BC b(b-1)/a (pairs inside B,
    each joined by a shortest paths of length 2, one through each A vertex)."""
    out = oracle_lib.bc(G.complete_bipartite(a, b))["bc"]
    assert _close(out[:a], b * (b - 1) / a)
    assert _close(out[a:], a * (a - 1) / b)


def test_grid_sigma_binomial_and_overflow(oracle_lib):
    """k x k grid: lambda(corner, opposite corner) = C(2k-2, k-1). k=34 fits in
    64 bits; k=35 does not, and the oracle must flag it."""
    for k in (2, 5, 12, 34, 35):
        g = G.grid_graph(k)
        row = oracle_lib.source(g, 0, with_delta=False)
        want = math.comb(2 * k - 2, k - 1)
        got = int(row["sigma"][-1]) | (int(row["sigma_hi"][-1]) << 64)
        assert got == want
        assert row["dist"][-1] == 2 * k - 2
        assert bool(row["flags"] & 1) == (want >= 1 << 64), k


def test_grid_uniform_weight_scales_distance(oracle_lib):
    """All weights c: same path counts, distances times c, same BC."""
    g1 = G.grid_graph(9)
    g3 = G.grid_graph(9, w=3)
    assert _close(oracle_lib.bc(g1)["bc"], oracle_lib.bc(g3)["bc"])
    for s in (0, 13, 40):
        r1 = oracle_lib.source(g1, s)
        r3 = oracle_lib.source(g3, s)
        assert np.array_equal(r1["sigma"], r3["sigma"])
        assert np.array_equal(r1["dist"] * 3, r3["dist"])


def test_layered_biclique_powers(oracle_lib):
    """Layer j of width w is reached by w^(j-1) shortest paths from vertex 0;
    width 16 crosses 2^64 at layer 17."""
    for width, layers in ((3, 6), (16, 17)):
        g = G.layered_biclique(layers, width)
        row = oracle_lib.source(g, 0, with_delta=False)
        for j in range(1, layers + 1):
            v = 1 + (j - 1) * width
            got = int(row["sigma"][v]) | (int(row["sigma_hi"][v]) << 64)
            assert got == width ** (j - 1)
            assert row["dist"][v] == j
        assert bool(row["flags"] & 1) == (width ** (layers - 1) >= 1 << 64)


# ------------------------------------------------ other routes of the paper

def test_literal_path_count_overwrites_beyond_distance_two():
    """As printed, ComputePathCount overwrites settled pairs when Diam >= 3;
    the corrected mask does not."""
    g = G.path_graph(4)
    a = algebraic.adjacency_matrix(g)
    lam_true, dist = algebraic.path_count(a)
    assert np.all(lam_true == 1)
    lit = algebraic.path_count_literal(a, int(dist.max()))
    assert lit[0, 1] != 1
    # on a diameter-2 graph the two agree
    k = G.complete_bipartite(2, 3)
    a2 = algebraic.adjacency_matrix(k)
    l2, d2 = algebraic.path_count(a2)
    assert np.array_equal(algebraic.path_count_literal(a2, 2), l2)


@pytest.mark.parametrize("seed", range(6))
def test_algebraic_and_algorithm2_match_oracle(oracle_lib, seed):
    n = [30, 45, 60, 80, 100, 120][seed]
    g = G.random_small(n, 3.0 / n, 400 + seed)
    a = algebraic.adjacency_matrix(g)
    lam, dist = algebraic.path_count(a)
    assert np.array_equal(dist, np.where(algebraic.apsp_minplus(g) >= algebraic.INF, -1,
                                         algebraic.apsp_minplus(g)))
    out = oracle_lib.bc(g)
    for s in range(0, n, 7):
        row = oracle_lib.source(g, s, with_delta=False)
        assert np.array_equal(row["dist"], dist[s])
        assert np.array_equal(row["sigma"].astype(object), lam[s].astype(object) % (1 << 64))
    delta = algebraic.dependency(a, dist, lam)
    assert _close(algebraic.bc_from_dependency(delta), out["bc"], rel=1e-10, abs_=1e-9)
    assert _close(algebraic.algorithm2(dist, lam), out["bc"], rel=1e-10, abs_=1e-9)
    reach = (dist >= 0).sum(axis=1)
    assert _close(np.diag(delta), reach - 1, rel=1e-10, abs_=1e-9)


def test_algorithm2_weighted_matches_oracle(oracle_lib):
    for seed in range(4):
        g = G.random_small(9, 0.4, 500 + seed, wmax=3)
        ref = brute.betweenness(g)
        dist = np.array([[-1 if x is None else x for x in row] for row in ref["dist"]])
        lam = np.array(ref["lam"], dtype=object)
        assert _close(algebraic.algorithm2(dist, lam), oracle_lib.bc(g)["bc"])


# ------------------------------------------------ directed graphs (Section 2)

@pytest.mark.parametrize("seed", range(8))
def test_directed_random_against_enumeration(oracle_lib, seed):
    """Directed graphs take P_s(v) over v's in-arcs (Section 1.1's definition
    with (u, v) an arc): the oracle against enumeration of the shortest
    directed paths, unweighted and with weights in {1, 2, 3}."""
    g = G.directed_random(8, 0.3, 700 + seed, wmax=0 if seed % 2 == 0 else 3)
    _check_against_brute(oracle_lib, g)


def test_directed_raw_enumeration(oracle_lib):
    g = G.directed_random(6, 0.4, 77, wmax=2)
    _check_against_brute(oracle_lib, g, brute.all_simple_paths_min(g))


@pytest.mark.parametrize("n", [2, 5, 12])
def test_directed_path_and_cycle(oracle_lib, n):
    """One-way path: vertex i is inside the unique path of the pairs
    s < i < t, so BC(i) = i(n-1-i). One-way cycle: at forward distance k
    (k = 2..n-1) each of the n pairs has k-1 inside vertices, so every vertex
    gets (n-1)(n-2)/2."""
    i = np.arange(n)
    assert _close(oracle_lib.bc(G.directed_path(n))["bc"], i * (n - 1 - i))
    assert _close(oracle_lib.bc(G.directed_cycle(n))["bc"], np.full(n, (n - 1) * (n - 2) / 2))


@pytest.mark.parametrize("n", [1, 2, 3, 6, 10])
def test_kkp_tripartite(oracle_lib, n):
    """Section 2's directed tripartite graph, weighted so that every shortest
    u_i - w_k path goes through v_0: the betweenness of v_0 is n^2 and every
    other vertex's is 0."""
    g = G.kkp_tripartite(n)
    want = np.zeros(3 * n)
    want[n] = n * n
    assert _close(oracle_lib.bc(g)["bc"], want)
    if n <= 3:
        _check_against_brute(oracle_lib, g)


def test_directed_algorithm2_matches_oracle(oracle_lib):
    for seed in range(3):
        g = G.directed_random(9, 0.3, 800 + seed, wmax=3)
        ref = brute.betweenness(g)
        dist = np.array([[-1 if x is None else x for x in row] for row in ref["dist"]])
        lam = np.array(ref["lam"], dtype=object)
        assert _close(algebraic.algorithm2(dist, lam), oracle_lib.bc(g)["bc"])


def test_undirected_given_as_directed(oracle_lib):
    """An undirected graph given as a directed one with both arcs of every
    edge has the same betweenness (its transpose is itself)."""
    g = G.random_small(30, 0.15, 901, connect=True, wmax=4)
    src = np.repeat(np.arange(g.n), g.degrees())
    d = G.csr_from_arcs(g.n, src, g.col, g.w)
    assert d.directed and np.array_equal(d.col, g.col)
    assert _close(oracle_lib.bc(d)["bc"], oracle_lib.bc(g)["bc"])


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(4))
def test_invariants_unweighted(oracle_lib, seed):
    g = G.random_small(70, 0.05, 600 + seed, connect=seed % 2 == 0)
    out = oracle_lib.bc(g)
    bc = out["bc"]
    assert np.all(bc >= -1e-12)
    # sum_v BC(v) = sum over ordered reachable pairs of (d(s,t) - 1)
    assert _close(bc.sum(), float((out["dist_sum"] - (out["reach"] - 1)).sum()), rel=1e-12)
    assert np.all(bc[g.degrees() == 1] == 0)
    for s in (0, 17, 33):
        row = oracle_lib.source(g, s)
        d = row["dist"]
        r = d >= 0
        # sum_{v != s} delta_s*(v) = sum_t (d(s,t) - 1)
        dv = row["delta"].copy()
        dv[s] = 0
        assert _close(dv.sum(), float((d[r] - 1).sum() + 1), rel=1e-12)
        # the shortest-path DAG of BFS joins levels that differ by at most one
        src = np.repeat(np.arange(g.n), g.degrees())
        both = r[src] & r[g.col]
        assert np.all(np.abs(d[src][both] - d[g.col][both]) <= 1)
        # Lemma 3.3: nothing depends on the farthest vertices
        far = d == d.max()
        assert np.all(row["delta"][far] == 0)
        # symmetry lambda_st = lambda_ts
        for t in np.nonzero(r)[0][:5]:
            back = oracle_lib.source(g, int(t), with_delta=False)
            assert back["sigma"][s] == row["sigma"][t] and back["dist"][s] == d[t]


def test_hashes_and_thread_count(oracle_lib):
    g = G.er_hamiltonian(300, 900, 77)
    one = oracle_lib.bc(g, threads=1)
    four = oracle_lib.bc(g, threads=4)
    assert _close(one["bc"], four["bc"], rel=1e-12)
    assert np.array_equal(one["hash_sigma"], four["hash_sigma"])
    v1 = np.arange(1, g.n + 1, dtype=np.uint64)
    for s in (0, 5, 299):
        row = oracle_lib.source(g, s, with_delta=False)
        with np.errstate(over="ignore"):
            hs = np.sum(row["sigma"] * v1, dtype=np.uint64)
            r = row["dist"] >= 0
            hd = np.sum((row["dist"][r] + 1).astype(np.uint64) * v1[r], dtype=np.uint64)
        assert hs == one["hash_sigma"][s] and hd == one["hash_dist"][s]
        assert one["arcs"][s] == row["arcs"]
    sub = oracle_lib.bc(g, sources=np.array([5, 0, 299], np.int32))
    assert sub["hash_sigma"][1] == one["hash_sigma"][0]


def test_rejects_bad_input(oracle_lib):
    g = G.path_graph(4)
    with pytest.raises(ValueError):
        oracle_lib.bc(g, sources=np.array([7], np.int32))
    bad = G.Graph(2, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), None)  # self-loop
    with pytest.raises(ValueError):
        oracle_lib.bc(bad)


# ---- the shortest-path DAG size (arcs (u, v) with u in P_s(v), Section 1.1),
# which the roofline's algorithmic bytes count: closed forms and a count from
# Floyd-Warshall distances that shares nothing with the oracle's BFS/Dijkstra.

def _dag_arcs_from_distances(g, s):
    d = brute.floyd_warshall(g)[s]
    adj = brute.adjacency(g)
    return sum(1 for u in range(g.n) if d[u] != brute.INF
               for v, w in adj[u] if d[v] != brute.INF and d[u] + w == d[v])


@pytest.mark.parametrize("n", [2, 5, 17])
def test_dag_arcs_path_star_complete(oracle_lib, n):
    # every one of these is a shortest-path tree from any source: n - 1 arcs
    for g, srcs in ((G.path_graph(n), (0, n // 2, n - 1)), (G.star_graph(n), (0, n - 1)),
                    (G.complete_graph(n), (0, n - 1))):
        for s in srcs:
            assert oracle_lib.source(g, s, with_delta=False)["arcs"] == n - 1, (g.name, s)
    # an odd cycle is a tree from every vertex; an even one adds the second
    # arc into the antipode
    assert oracle_lib.source(G.cycle_graph(2 * n + 1), 3, with_delta=False)["arcs"] == 2 * n
    assert oracle_lib.source(G.cycle_graph(2 * n), 3, with_delta=False)["arcs"] == 2 * n


@pytest.mark.parametrize("a,b", [(1, 4), (3, 5), (6, 2)])
def test_dag_arcs_complete_bipartite(oracle_lib, a, b):
    # from an A vertex: b arcs to the B side, then each of the other a - 1 A
    # vertices has all b B vertices as predecessors; from a B vertex the roles swap
    g = G.complete_bipartite(a, b)
    assert oracle_lib.source(g, 0, with_delta=False)["arcs"] == b + (a - 1) * b
    assert oracle_lib.source(g, a, with_delta=False)["arcs"] == a + (b - 1) * a


@pytest.mark.parametrize("k", [2, 5, 9])
def test_dag_arcs_grid_corner(oracle_lib, k):
    # from a corner every vertex (i, j) has predecessors (i-1, j) and (i, j-1)
    # where they exist: 2 k (k - 1) arcs; uniform weights change nothing
    assert oracle_lib.source(G.grid_graph(k), 0, with_delta=False)["arcs"] == 2 * k * (k - 1)
    assert oracle_lib.source(G.grid_graph(k, 7), 0, with_delta=False)["arcs"] == 2 * k * (k - 1)


@pytest.mark.parametrize("seed", range(4))
def test_dag_arcs_against_distance_table(oracle_lib, seed):
    for g in (G.random_small(11, 0.35, 600 + seed), G.random_small(10, 0.4, 700 + seed, wmax=3)):
        out = oracle_lib.bc(g)
        for s in range(g.n):
            want = _dag_arcs_from_distances(g, s)
            assert oracle_lib.source(g, s, with_delta=False)["arcs"] == want, (g.name, s)
            assert out["arcs"][s] == want
