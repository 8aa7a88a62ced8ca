"""bc_run_noalloc: the entry point for callers that cannot allocate device
memory (a pool or custom allocator owns the GPU, or allocation is forbidden
after start-up). Its scratch is one fixed __device__ array shared by every
call, so each graph here is run through it twice in a row, and both results
are compared with the CPU oracle and with bc_run, within the tolerance the
other GPU tests use. Its own limits are pinned too: the deepest BFS it takes,
the first one it refuses, and ids out of range. This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0809_1906_gb300 import graphs as G

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _close(got, ref, n):
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * max(n, 1))
    return np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref))) if n else 0.0


def _noalloc(lib, g, src=None, n=None):
    """One bc_run_noalloc call on device copies of g; returns (status, bc)."""
    import torch
    stream = torch.cuda.current_stream()
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda() if g.col.size else torch.zeros(1, dtype=torch.int32, device="cuda")
    s = None if src is None else torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda()
    out = torch.full((max(g.n, 1),), float("nan"), dtype=torch.float64, device="cuda")
    code = lib.bc_run_noalloc(g.n if n is None else n, _ptr(rp), _ptr(col), _ptr(s),
                              0 if s is None else int(s.numel()), _ptr(out), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return code, out[: g.n].cpu().numpy()


def test_noalloc_matches_oracle_and_bc_run_twice_in_a_row():
    from paper_0809_1906_gb300 import native
    lib = native.load()
    graphs = [(G.er_hamiltonian(1500, 6000, 41), None),
              (G.random_small(700, 3.0 / 700, 42, connect=False), G.sample_sources(700, 300, 43)),
              (G.er_hamiltonian(16384, 60000, 44), G.sample_sources(16384, 200, 45))]
    for g, src in graphs:
        ref = oracle.bc(g, src)["bc"]
        via_run, _ = native.betweenness(g, src)
        for call in range(2):  # the second call finds the first one's scratch contents
            code, got = _noalloc(lib, g, src)
            assert code == native.BC_OK, lib.bc_status_string(code)
            ok, worst = _close(got, ref, g.n)
            assert ok, (g.name, call, "vs oracle", worst)
            ok, worst = _close(got, via_run, g.n)
            assert ok, (g.name, call, "vs bc_run", worst)


def test_noalloc_deepest_accepted_bfs_and_first_refused():
    """P_63 from its ends is 62 levels deep, the most the scratch holds:
    BC(v_i) = 2(i-1)(n-i) over ordered pairs. P_64 is one level deeper."""
    from paper_0809_1906_gb300 import native
    lib = native.load()
    g = G.path_graph(63)
    i = np.arange(1, 64, dtype=np.float64)
    for _ in range(2):
        code, got = _noalloc(lib, g)
        assert code == native.BC_OK
        assert np.allclose(got, 2 * (i - 1) * (63 - i), rtol=1e-6, atol=1e-6)
    code, _ = _noalloc(lib, G.path_graph(64))
    assert code == native.BC_ERR_UNSUPPORTED
    code, _ = _noalloc(lib, G.path_graph(64), np.array([1, 62], np.int32))  # depth 62 from these two
    assert code == native.BC_OK


def test_noalloc_rejects_bad_ids_and_sizes():
    from paper_0809_1906_gb300 import native
    lib = native.load()
    g = G.path_graph(10)
    code, _ = _noalloc(lib, g, np.array([0, 10], np.int32))  # source id n, found by the device check
    assert code == native.BC_ERR_ARG
    code, _ = _noalloc(lib, g, np.array([-1], np.int32))
    assert code == native.BC_ERR_ARG
    bad = G.Graph(3, np.array([0, 1, 2, 3], np.int32), np.array([1, 3, 1], np.int32), None)  # neighbour id 3
    code, _ = _noalloc(lib, bad)
    assert code == native.BC_ERR_ARG
    code, got = _noalloc(lib, g)  # a valid call right after the refused ones
    i = np.arange(1, 11, dtype=np.float64)
    assert code == native.BC_OK and np.allclose(got, 2 * (i - 1) * (10 - i), rtol=1e-6)
    import torch
    n = 16385  # one past BC_NOALLOC_MAX_N
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    assert lib.bc_run_noalloc(n, _ptr(rp), _ptr(rp), None, 0, _ptr(out), None) == native.BC_ERR_ARG
