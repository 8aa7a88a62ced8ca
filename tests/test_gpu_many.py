"""GPU parity of the many-graph persistent launch against the oracle."""
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


def close(got, ref, n):
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * max(n, 1))
    return np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("batch", [32, 64, 128, 256])
def test_many_small_graphs(nat, batch):
    gs = G.many_graphs(40, 20, 600, seed=77)
    gs.append(G.path_graph(100))  # deeper than the 64-level capacity: re-run path
    gs.append(G.csr_from_edges(1, [], []))
    hs = [nat.Graph.from_csr(g) for g in gs]
    try:
        with nat.ManyPlan(hs, batch=batch) as plan:
            for rep in range(2):  # replay of the captured graph
                plan.run()
                code, flags, rerun = plan.result()
                assert code == nat.BC_OK and rerun == 1
                for g, h in zip(gs, hs):
                    got, _, _ = h.result()
                    assert close(got, oracle.bc(g)["bc"], g.n), (g.name, rep)
    finally:
        for h in hs:
            h.close()


def test_many_split_graph_deterministic(nat):
    """One large graph among small ones is split into several items whose
    partials are added in item order: two runs give identical bits."""
    gs = [G.er_hamiltonian(3000, 9000, 5)] + G.many_graphs(10, 20, 80, seed=3)
    hs = [nat.Graph.from_csr(g) for g in gs]
    try:
        with nat.ManyPlan(hs) as plan:
            plan.run()
            plan.result()
            a, _, _ = hs[0].result()
            plan.run()
            plan.result()
            b, _, _ = hs[0].result()
        assert np.array_equal(a, b)
        assert close(a, oracle.bc(gs[0])["bc"], gs[0].n)
    finally:
        for h in hs:
            h.close()
