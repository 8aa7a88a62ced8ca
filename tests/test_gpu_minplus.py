"""GPU parity of the weighted algebraic path (BC_DENSE on a weighted graph):
distance products with path counts (Section 3.2) bit-exact against the
oracle's rows, and BC through Algorithm 2's pair formula within
max(1e-5 |ref|, 1e-6 n)."""
import ctypes
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


def dense_rows(nat, g, src):
    src = np.ascontiguousarray(src, np.int32)
    sig = np.empty((src.size, g.n), np.uint64)
    dist = np.empty((src.size, g.n), np.int32)
    with nat.Graph.from_csr(g) as h:
        opt = nat.make_options(0, nat.BC_DENSE)
        code = h.lib.bc_forward_rows(h.handle, nat._addr(src), int(src.size), nat._addr(sig), nat._addr(dist),
                                     ctypes.byref(opt), nat._stream_ptr(None))
    return sig, dist, code


def check_rows(nat, g, src):
    sig, dist, code = dense_rows(nat, g, src)
    assert code >= 0
    for i, s in enumerate(np.asarray(src).tolist()):
        o = oracle.source(g, s, with_delta=False)
        assert np.array_equal(dist[i], o["dist"].astype(np.int32)), (g.name, s)
        assert np.array_equal(sig[i], o["sigma"]), (g.name, s)
    return code


def check_bc(nat, g):
    ref = oracle.bc(g)
    with nat.Graph.from_csr(g) as h:
        h.run(flags=nat.BC_DENSE)
        got, code, _ = h.result()
        hs = h.source_hashes(g.n)
    tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
    assert np.all(np.abs(got - ref["bc"]) <= tol), (g.name, float(np.max(np.abs(got - ref["bc"]))))
    for k in ("hash_sigma", "hash_dist", "dist_sum", "reach"):
        assert np.array_equal(hs[k], ref[k]), (g.name, k)
    return got


@pytest.mark.parametrize("n,p,wmax,seed", [(70, 0.1, 3, 1), (200, 0.05, 9, 2), (513, 0.02, 100, 3)])
def test_rows_random_weighted(nat, n, p, wmax, seed):
    """Ragged sizes (n and the source count not multiples of the 64 x 64
    tiles); several steps of the product before nothing changes."""
    g = G.random_small(n, p, 1400 + seed, wmax=wmax, connect=seed != 2)
    src = G.sample_sources(n, min(n, 97), 3 + seed)
    check_rows(nat, g, src)


def test_rows_grid_deep_and_overflow(nat):
    """Unit weights on a 35 x 35 grid (given as a weighted graph): 68 steps of
    the product; sigma(corner, far corner) = C(68,34) >= 2^64 wraps and sets
    the overflow warning."""
    g0 = G.grid_graph(35)
    g = G.Graph(g0.n, g0.row_ptr, g0.col, np.ones_like(g0.col), "grid35w")
    sig, dist, code = dense_rows(nat, g, np.array([0], np.int32))
    assert code == nat.BC_WARN_SIGMA_OVERFLOW
    assert int(sig[0, -1]) == math.comb(68, 34) % (1 << 64) and dist[0, -1] == 68


@pytest.mark.parametrize("seed", range(3))
def test_bc_random_weighted(nat, seed):
    check_bc(nat, G.random_small(300 + 50 * seed, 0.03, 1500 + seed, wmax=5, connect=seed % 2 == 0))


def test_bc_directed_weighted_and_kkp(nat):
    check_bc(nat, G.directed_random(250, 0.03, 1600, wmax=6))
    got = check_bc(nat, G.kkp_tripartite(20))
    assert abs(got[20] - 400.0) <= 1e-6 * 400


def test_bc_matches_weighted_sweep(nat):
    """Two GPU routes on one weighted graph: the bucket kernel's backward
    sweep and distance products + pair formula."""
    g = G.random_small(600, 0.02, 1700, wmax=20)
    with nat.Graph.from_csr(g) as h:
        h.run()
        a, _, _ = h.result()
        h.run(flags=nat.BC_DENSE)
        b, _, _ = h.result()
    assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * g.n)


def test_rejects_source_subset(nat):
    g = G.random_small(50, 0.1, 1800, wmax=3)
    with nat.Graph.from_csr(g) as h:
        with pytest.raises(nat.BcError) as e:
            h.run(np.arange(10, dtype=np.int32), flags=nat.BC_DENSE)
        assert e.value.code == nat.BC_ERR_ARG
