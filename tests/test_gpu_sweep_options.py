"""GPU tests of the level-sweep options: the direction of the first level
(top-down push or bottom-up pull, by the alpha rule or forced), the
look-ahead's tail threshold, and the bounded waits' timeout paths (host and
device), each against the CPU oracle."""
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


def _close(got, ref, n):
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * max(n, 1))
    return np.all(np.abs(got - ref) <= tol)


GRAPHS = [G.er_hamiltonian(2000, 7000, 91), G.random_small(900, 2.2 / 900, 92, connect=False),
          G.grid_graph(20), G.path_graph(150), G.star_graph(300)]


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("batch,chunk", [(64, 8), (256, 0)])
def test_first_level_direction_and_tail(nat, g, batch, chunk):
    """Top-down or bottom-up at level 0 -> 1 (alpha tiny: always top-down;
    alpha huge or BC_FORCE_BOTTOMUP: bottom-up) and any tail threshold give
    the same exact sigma/distance summaries and DAG arcs as the oracle, and BC
    identical to the bit (the direction changes how level 1 is found, never
    what it holds; the sums over it run in the same order)."""
    ref = oracle.bc(g)
    outs = []
    with nat.Graph.from_csr(g) as h:
        for alpha, beta, flags in ((1e-6, 0.0, 0), (1e6, 0.5, 0), (0.0, 1.0, nat.BC_FORCE_BOTTOMUP), (0.0, 0.0, 0)):
            h.run(batch=batch, chunk=chunk, alpha=alpha, beta=beta, flags=flags)
            got, code, _ = h.result()
            hs = h.source_hashes(g.n)
            arcs, _ = h.run_stats()
            assert code == nat.BC_OK
            assert _close(got, ref["bc"], g.n), (g.name, alpha, beta, flags)
            for k in ("hash_sigma", "hash_dist", "dist_sum", "reach"):
                assert np.array_equal(hs[k], ref[k]), (g.name, alpha, beta, flags, k)
            assert arcs == int(ref["arcs"].sum())
            outs.append(got)
    # the level-1 counts (top-down) and the rows (bottom-up) differ in form,
    # so BC may differ in its last FP32 bits between directions, not within one
    assert np.array_equal(outs[0], outs[3])


def test_bottom_up_first_level_rows(nat):
    g = G.er_hamiltonian(1200, 5000, 93)
    with nat.Graph.from_csr(g) as h:
        sig, dist, _ = h.forward_rows(np.array([0, 7, 1199], np.int32), batch=32,
                                      flags=nat.BC_FORCE_BOTTOMUP)
    for i, s in enumerate((0, 7, 1199)):
        o = oracle.source(g, s, with_delta=False)
        assert np.array_equal(sig[i], o["sigma"]) and np.array_equal(dist[i], o["dist"].astype(np.int32))


def test_unsupported_bucket_width(nat):
    g = G.grid_graph(5, 3)
    with nat.Graph.from_csr(g) as h:
        with pytest.raises(nat.BcError) as e:
            h.run(delta=4)
        assert e.value.code == nat.BC_ERR_UNSUPPORTED
        h.run(delta=1)
        got, _, _ = h.result()
    assert _close(got, oracle.bc(g)["bc"], g.n)


def test_host_wait_limit_expires_then_next_run_is_correct(nat):
    """A 1 ms host wait limit on a BFS thousands of levels deep: bc_run gives
    up with BC_ERR_TIMEOUT (the kernels it launched finish on their own);
    after a device synchronisation the same handle runs correctly."""
    import torch
    g = G.path_graph(3000)
    with nat.Graph.from_csr(g) as h:
        with pytest.raises(nat.BcError) as e:
            h.run(np.arange(0, 3000, 97, dtype=np.int32), batch=32, wait_limit_ms=1)
        assert e.value.code == nat.BC_ERR_TIMEOUT
        torch.cuda.synchronize()
        src = np.array([0, 1500, 2999], np.int32)
        h.run(src, batch=32)
        got, code, _ = h.result()
    assert code == nat.BC_OK and _close(got, oracle.bc(g, src)["bc"], g.n)


def test_device_wait_expiry_reports_timeout_then_next_run_is_correct(nat):
    """With the test hook every staged-row wait also expects bytes that never
    arrive, so each wait runs out after 50 us: the warps release those bytes,
    wait for their own copies, stop staging, and bc_result reports
    BC_ERR_TIMEOUT with the copy-timeout status bit. The context stays usable:
    the next run on the same handle matches the oracle."""
    g = G.er_hamiltonian(3000, 12000, 94)
    ref = oracle.bc(g)
    with nat.Graph.from_csr(g) as h:
        h.run(batch=256, flags=nat.BC_TEST_WAIT_EXPIRY, device_wait_us=50)
        with pytest.raises(nat.BcError) as e:
            h.result()
        assert e.value.code == nat.BC_ERR_TIMEOUT
        h.run(batch=256)
        got, code, st = h.result()
        assert code == nat.BC_OK and st == 0
        assert _close(got, ref["bc"], g.n)


def test_run_log_lines(nat, tmp_path):
    """BC_LOG=1: every bc_result writes one JSON line with the run's sizes,
    options and host wall time (a fresh process, since the library reads the
    variable once)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_0809_1906_gb300 import graphs as G, native\n"
            "g = G.er_hamiltonian(500, 2000, 95)\n"
            "with native.Graph.from_csr(g) as h:\n"
            "    h.run(batch=64); h.result(); h.run(batch=128, beta=0.25); h.result()\n") % root
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, BC_LOG="1"), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [json.loads(x) for x in r.stderr.splitlines() if x.startswith('{"bc_log"')]
    assert len(lines) == 2
    assert lines[0]["n"] == 500 and lines[0]["batch"] == 64 and lines[1]["batch"] == 128
    assert abs(lines[1]["beta"] - 0.25) < 1e-6 and lines[1]["sources"] == 500 and lines[1]["status"] == 0
    assert lines[0]["wall_ms"] > 0 and lines[0]["launches"] > 0
