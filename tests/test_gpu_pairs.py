"""GPU parity of BC_PAIRS: betweenness from all-pairs rows with Algorithm 2's
pair formula (Section 4.2.1), against the oracle and against the level
sweep on the same graphs. Tolerance max(1e-5 |ref|, 1e-6 n)."""
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


def pairs_bc(nat, g, **run):
    with nat.Graph.from_csr(g) as h:
        h.run(flags=nat.BC_PAIRS | run.pop("flags", 0), **run)
        got, code, _ = h.result()
        hs = h.source_hashes(g.n)
    return got, code, hs


def check(nat, g):
    ref = oracle.bc(g)
    got, code, hs = pairs_bc(nat, g)
    tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
    assert np.all(np.abs(got - ref["bc"]) <= tol), (g.name, float(np.max(np.abs(got - ref["bc"]))))
    assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]) and np.array_equal(hs["hash_dist"], ref["hash_dist"])
    assert code == nat.BC_OK
    return got


@pytest.mark.parametrize("g", [G.path_graph(2), G.path_graph(17), G.cycle_graph(13), G.star_graph(30),
                               G.complete_graph(12), G.complete_bipartite(3, 5), G.grid_graph(8)],
                         ids=lambda g: g.name)
def test_closed_form_graphs(nat, g):
    check(nat, g)


@pytest.mark.parametrize("n,p,seed", [(100, 0.05, 1), (300, 0.02, 2), (1000, 0.01, 3)])
def test_random_unweighted_ragged(nat, n, p, seed):
    """n not a multiple of the 32 x 64 tiles; every other seed disconnected."""
    check(nat, G.random_small(n, p, 1100 + seed, connect=seed % 2 == 1))


@pytest.mark.parametrize("seed", range(2))
def test_random_weighted(nat, seed):
    check(nat, G.random_small(500, 0.01, 1200 + seed, wmax=7))


def test_directed_and_kkp(nat):
    check(nat, G.directed_random(400, 0.02, 1300))
    check(nat, G.directed_random(300, 0.02, 1301, wmax=4))
    got = check(nat, G.kkp_tripartite(30))
    assert abs(got[30] - 900.0) <= 1e-6 * 900


def test_pairs_equal_level_sweep(nat):
    """Two GPU routes to BC on the same graph: the pair formula and the
    backward sweep of Theorem 1.1."""
    g = G.er_hamiltonian()
    with nat.Graph.from_csr(g) as h:
        h.run()
        a, _, _ = h.result()
        h.run(flags=nat.BC_PAIRS)
        b, _, _ = h.result()
    assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * g.n)


def test_pairs_argument_checks(nat):
    g = G.path_graph(40)
    with nat.Graph.from_csr(g) as h:
        with pytest.raises(nat.BcError) as e:
            h.run(np.arange(5, dtype=np.int32), flags=nat.BC_PAIRS)
        assert e.value.code == nat.BC_ERR_ARG
        with pytest.raises(nat.BcError):
            h.run(flags=nat.BC_PAIRS | nat.BC_PLAIN)
