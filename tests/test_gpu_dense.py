"""GPU parity of the tensor-core level expansion (BC_DENSE) against the
oracle: sigma and distances bit-exact through the limb split and carry
combine, BC within tolerance."""
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


def check(nat, g, sources=None, rows=16):
    ref = oracle.bc(g, sources)
    with nat.Graph.from_csr(g) as h:
        h.run(sources, flags=nat.BC_DENSE)
        got, code, _ = h.result()
        ns = g.n if sources is None else len(sources)
        hs = h.source_hashes(ns)
        assert np.array_equal(hs["hash_sigma"], ref["hash_sigma"]), g.name
        assert np.array_equal(hs["hash_dist"], ref["hash_dist"]), g.name
        tol = np.maximum(1e-5 * np.abs(ref["bc"]), 1e-6 * g.n)
        assert np.all(np.abs(got - ref["bc"]) <= tol), (g.name, float(np.max(np.abs(got - ref["bc"]))))
        assert code == (nat.BC_WARN_SIGMA_OVERFLOW if ref["flags"] & 1 else nat.BC_OK)
        if rows:
            src = np.arange(g.n, dtype=np.int32) if sources is None else np.asarray(sources, np.int32)
            pick = src[:rows]
            with nat.Graph.from_csr(g) as h2:
                import ctypes
                sig = np.empty((pick.size, g.n), np.uint64)
                dist = np.empty((pick.size, g.n), np.int32)
                opt = nat.make_options(0, nat.BC_DENSE)
                nat._check(h2.lib.bc_forward_rows(h2.handle, nat._addr(pick), int(pick.size), nat._addr(sig),
                                                  nat._addr(dist), ctypes.byref(opt), nat._stream_ptr(None)),
                           "bc_forward_rows")
            for i, s in enumerate(pick.tolist()):
                o = oracle.source(g, s, with_delta=False)
                assert np.array_equal(dist[i], o["dist"].astype(np.int32)), (g.name, s)
                assert np.array_equal(sig[i], o["sigma"]), (g.name, s)


def test_dense_small_random(nat):
    """n = 256 (4 tensor-core tiles), one batch of 128 sources."""
    g = G.gnp(256, 0.05, seed=11)
    check(nat, g, sources=np.arange(128, dtype=np.int32))


@pytest.mark.parametrize("n,p", [(100, 0.1), (300, 0.02), (1000, 0.01)])
def test_dense_ragged_and_deep(nat, n, p):
    """n not a multiple of 64 (padding), several levels, ragged last batch."""
    g = G.random_small(n, p, 70 + n, connect=True)
    check(nat, g)


def test_dense_multi_limb_and_overflow(nat):
    """Layered bicliques: counts w^j need several 8-bit limbs and carries;
    width 16 over 17 layers reaches 2^64 (flagged, low 64 bits exact)."""
    check(nat, G.layered_biclique(6, 9))
    g = G.layered_biclique(17, 16)
    with nat.Graph.from_csr(g) as h:
        import ctypes
        src = np.array([0], np.int32)
        sig = np.empty((1, g.n), np.uint64)
        dist = np.empty((1, g.n), np.int32)
        opt = nat.make_options(0, nat.BC_DENSE)
        code = h.lib.bc_forward_rows(h.handle, nat._addr(src), 1, nat._addr(sig), nat._addr(dist), ctypes.byref(opt),
                                     nat._stream_ptr(None))
    o = oracle.source(g, 0, with_delta=False)
    assert code == nat.BC_WARN_SIGMA_OVERFLOW
    assert np.array_equal(sig[0], o["sigma"]) and np.array_equal(dist[0], o["dist"].astype(np.int32))


def test_dense_gnp8192(nat):
    """G(8192, 0.05): the dense configuration. All sources in 64 batches of
    128 (the benchmark's launch configuration); per-source hashes on a sample
    and BC over one batch against the oracle."""
    g = G.gnp(8192, 0.05)
    with nat.Graph.from_csr(g) as h:
        h.run(flags=nat.BC_DENSE)
        bc, code, _ = h.result()
        hs = h.source_hashes(g.n)
        assert code == nat.BC_OK
        pick = G.sample_sources(g.n, 24, 5)
        ref = oracle.bc(g, pick)
        assert np.array_equal(hs["hash_sigma"][pick], ref["hash_sigma"])
        assert np.array_equal(hs["hash_dist"][pick], ref["hash_dist"])
        rhs = float((hs["dist_sum"] - (hs["reach"] - 1)).sum())
        assert abs(bc.sum() - rhs) <= 1e-6 * rhs
        sub = np.arange(128, dtype=np.int32)
        h.run(sub, flags=nat.BC_DENSE)
        got, _, _ = h.result()
        r = oracle.bc(g, sub)["bc"]
        assert np.all(np.abs(got - r) <= np.maximum(1e-5 * np.abs(r), 1e-6 * g.n))


@pytest.mark.parametrize("n,p", [(256, 0.05), (700, 0.006), (1000, 0.01)])
def test_dense_backward_tensor_vs_sparse(nat, n, p):
    """The tensor-core backward (three bf16 parts of the FP32 c rows) agrees
    with the sparse backward and with the oracle; deeper graphs exercise the
    alternating split-row blocks over several levels."""
    g = G.random_small(n, p, 90 + n, connect=True)
    ref = oracle.bc(g)["bc"]
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * g.n)
    with nat.Graph.from_csr(g) as h:
        h.run(flags=nat.BC_DENSE)
        a, _, _ = h.result()
        h.run(flags=nat.BC_DENSE | nat.BC_SPARSE_BACKWARD)
        b, _, _ = h.result()
    assert np.all(np.abs(a - ref) <= tol), float(np.max(np.abs(a - ref) / np.maximum(np.abs(ref), 1)))
    assert np.all(np.abs(b - ref) <= tol)


def test_dense_limb_sums_stay_exact(nat):
    """Source 0 -> 15 vertices -> 2000 vertices joined to all 15 (sigma 15 each)
    -> one vertex joined to all 2000: its count 15 * 2000 = 30000 is one limb
    product's sum of 2000 terms of 15, which needs about 15 significant bits
    of the tensor core's accumulator (so does every 4-bit-limb or 8-bit-limb
    level here). sigma and d bit-exact from every source, BC within bounds."""
    a, b = 15, 2000
    L1 = np.arange(1, 1 + a)
    L2 = np.arange(1 + a, 1 + a + b)
    top = 1 + a + b
    us = [np.zeros(a, np.int64), np.repeat(L1, b), L2]
    vs = [L1, np.tile(L2, a), np.full(b, top)]
    g = G.csr_from_edges(top + 1, np.concatenate(us), np.concatenate(vs), name="fan_15_2000")
    src = np.ascontiguousarray(np.arange(g.n, dtype=np.int32)[::7])  # includes source 0
    check(nat, g, sources=src, rows=4)


def test_dense_tensor_work_by_operand_type(nat):
    """The forward's limb products run in e4m3 while a level's counts fit four
    4-bit limbs, the backward's in bf16: bc_run_stats reports each. Level 1
    -> 2 of G(300, 0.05) has all counts 1 (one e4m3 limb); the sparse
    backward issues no bf16 work."""
    g = G.gnp(300, 0.05, seed=3)
    with nat.Graph.from_csr(g) as h:
        h.run(flags=nat.BC_DENSE)
        h.result()
        bf, f8 = h.dense_flops_by_type()
        npad = 384
        assert f8 >= 2.0 * 128 * npad * npad * 3  # at least one e4m3 level for each of the 3 batches
        assert bf >= 2.0 * 128 * 3 * npad * npad  # at least one bf16 backward level (3 parts)
        assert h.dense_flops() == bf + f8
        h.run(flags=nat.BC_DENSE | nat.BC_SPARSE_BACKWARD)
        h.result()
        bf2, f82 = h.dense_flops_by_type()
        assert bf2 == 0.0 and f82 == f8
