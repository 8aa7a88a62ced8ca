"""bc_run_noalloc: the entry point for callers that cannot allocate device
memory (a pool or custom allocator owns the GPU, or allocation is forbidden
after start-up). Its scratch is one fixed __device__ array shared by every
call, so it is checked here on two calls in a row against bc_run, within the
tolerance the other GPU tests use. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_0809_1906_gb300 import graphs as G

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_matches_bc_run_twice_in_a_row():
    import torch
    from paper_0809_1906_gb300 import native
    lib = native.load()
    stream = torch.cuda.current_stream()
    graphs = [(G.er_hamiltonian(1500, 6000, 41), None),
              (G.random_small(700, 3.0 / 700, 42, connect=False), G.sample_sources(700, 300, 43))]
    for g, src in graphs:
        ref, _ = native.betweenness(g, src)
        rp = torch.from_numpy(g.row_ptr).cuda()
        col = torch.from_numpy(g.col).cuda()
        s = None if src is None else torch.from_numpy(np.ascontiguousarray(src, np.int32)).cuda()
        out = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
        code = lib.bc_run_noalloc(g.n, _ptr(rp), _ptr(col), _ptr(s), 0 if s is None else int(s.numel()),
                                  _ptr(out), ctypes.c_void_p(stream.cuda_stream))
        assert code == native.BC_OK, lib.bc_status_string(code)
        got = out.cpu().numpy()
        tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * g.n)
        assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref)))


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    from paper_0809_1906_gb300 import native
    lib = native.load()
    n = 16385  # one past BC_NOALLOC_MAX_N
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    code = lib.bc_run_noalloc(n, _ptr(rp), _ptr(rp), None, 0, _ptr(out), None)
    assert code == native.BC_ERR_ARG
