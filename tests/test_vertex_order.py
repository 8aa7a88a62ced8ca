"""CPU checks of bc_vertex_order, the numbering with locality that the weighted
sweep runs on (host code, no GPU)."""
import numpy as np
import pytest

from paper_0809_1906_gb300 import graphs as G
from paper_0809_1906_gb300 import native


def order(g):
    return native.vertex_order(g.n, g.row_ptr, g.col)


def is_perm(p, n):
    return p.shape == (n,) and np.array_equal(np.sort(p), np.arange(n, dtype=p.dtype))


def arcs(g):
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    return np.repeat(np.arange(g.n), np.diff(rp)), np.asarray(g.col, dtype=np.int64)


def test_permutation_on_assorted_graphs():
    graphs = [G.grid_graph(1), G.grid_graph(7), G.random_small(333, 0.01, 4, connect=False),
              G.random_small(50, 0.3, 5), G.rmat_lcc(scale=10, edge_factor=8), G.csr_from_edges(6, [], [], name="empty6")]
    for g in graphs:
        p = order(g)
        assert is_perm(p, g.n), g.name
        assert np.array_equal(p, order(g)), g.name  # deterministic
    assert order(G.csr_from_edges(0, [], [], name="none")).shape == (0,)


def test_star_and_isolated_vertices():
    n = 40
    star = G.csr_from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), name="star")
    p = order(star)
    assert is_perm(p, n)
    # the hub matches its first leaf; the other leaves stay alone, so the
    # coarsening stops after one level and keeps the id order otherwise
    assert p[0] == 0 and p[1] == 1 and np.array_equal(p[2:], np.arange(2, n))


def test_path_of_power_of_two_keeps_its_order():
    # id-order matching pairs (0,1), (2,3), ... at every level: the hierarchy
    # is the path's own order
    n = 64
    g = G.csr_from_edges(n, np.arange(n - 1), np.arange(1, n), name="path64")
    assert np.array_equal(order(g), np.arange(n))


def test_square_grid_becomes_nested_squares():
    # a 2^k x 2^k grid in row-major ids: level 1 pairs horizontal neighbours,
    # level 2 joins two dominoes along their two-edge side, and so on, so
    # every aligned block of 4^j new ids is a 2^j x 2^j square
    k = 16
    g = G.grid_graph(k)
    p = order(g)
    assert is_perm(p, k * k)
    r, c = np.divmod(np.argsort(p), k)  # position of new id i
    for size in (4, 16, 64):
        side = int(round(size ** 0.5))
        for b in range(0, k * k, size):
            rr, cc = r[b:b + size], c[b:b + size]
            assert rr.max() - rr.min() == side - 1 and cc.max() - cc.min() == side - 1, (size, b)
            assert rr.min() % side == 0 and cc.min() % side == 0, (size, b)


def test_shuffled_grid_regains_locality():
    g0 = G.grid_longrange(side=128, frac=0.05, wmax=10, seed=3)
    u, v, w = g0.edges()
    shuf = np.random.default_rng(0).permutation(g0.n)
    g = G.csr_from_edges(g0.n, shuf[u], shuf[v], w, name="shuffled")
    s, t = arcs(g)
    before = np.mean(np.abs(s - t) < 64)
    q = order(g).astype(np.int64)
    after = np.mean(np.abs(q[s] - q[t]) < 64)
    assert before < 0.01 and after > 0.6, (before, after)
    # the grid in its own row-major ids: most arcs end up within one 64-id run
    s0, t0 = arcs(g0)
    q0 = order(g0).astype(np.int64)
    assert np.mean(np.abs(q0[s0] - q0[t0]) < 64) > 0.8


@pytest.mark.parametrize("bad", ["rp0", "decreasing", "head", "null"])
def test_rejects_malformed_input(bad):
    g = G.grid_graph(5)
    rp = np.asarray(g.row_ptr, np.int32).copy()
    col = np.asarray(g.col, np.int32).copy()
    n = g.n
    if bad == "rp0":
        rp[0] = 1
    elif bad == "decreasing":
        rp[3] = rp[2] - 1
    elif bad == "head":
        col[7] = n
    elif bad == "null":
        col = np.zeros(0, np.int32)
    with pytest.raises(native.BcError) as e:
        native.vertex_order(n, rp, col)
    assert e.value.code == native.BC_ERR_ARG


def test_directed_and_irregular_csr():
    # the weighted sweep orders a directed graph by its out-arcs; self-loops
    # and repeated heads are accepted here (bc_create_graph rejects them)
    g = G.directed_random(300, 0.02, 7, wmax=3)
    p = order(g)
    assert is_perm(p, g.n) and np.array_equal(p, order(g))
    rp = np.array([0, 3, 4, 4, 6], np.int32)
    col = np.array([0, 1, 1, 0, 3, 3], np.int32)
    p = native.vertex_order(4, rp, col)
    assert is_perm(p, 4)
