"""What the toolchain allows on sm_103a for the algebraic path (no GPU: nvcc
and ptxas only). The 8-bit-integer tensor-core form (tcgen05.mma kind::i8,
u8 x u8 -> s32) assembles for sm_100a but not for sm_103a, so on GB300 the
limb products of Section 3.1.1 run as e4m3 x e4m3 -> FP32 (kind::f8f6f4; exact
for 4-bit limbs while 15 n < 2^24) or bf16 x bf16 -> FP32 (kind::f16; exact
for 8-bit limbs while 255 n < 2^24)."""
import os
import shutil
import subprocess

import pytest

PROBE = r'''
#include <cstdint>
__global__ void k(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
'''


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not available")


def _assemble(tmp_path, kind, arch):
    src = tmp_path / f"probe_{kind}_{arch}.cu"
    src.write_text(PROBE.replace("KIND", kind))
    r = subprocess.run([_nvcc(), "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", str(src),
                        "-o", str(tmp_path / "probe.o")], capture_output=True, text=True)
    return r.returncode, r.stdout + r.stderr


def test_integer_tensor_cores_are_not_available_on_sm103a(tmp_path):
    rc, out = _assemble(tmp_path, "i8", "103a")
    assert rc != 0 and "kind::i8" in out and "sm_103a" in out, out
    rc, out = _assemble(tmp_path, "i8", "100a")
    assert rc == 0, out
    rc, out = _assemble(tmp_path, "f16", "103a")  # the forms the dense path uses
    assert rc == 0, out
    rc, out = _assemble(tmp_path, "f8f6f4", "103a")
    assert rc == 0, out
