"""Which 8-bit tensor-core MMA kinds the toolchain assembles for sm_103a.

The dense path multiplies {0,1} operands held as e4m3 (tcgen05.mma
kind::f8f6f4) with fp32 accumulation; an int8 MMA with int32 accumulation
would be the textbook choice for counts.  ptxas assembles kind::i8 for
sm_100a but refuses it for sm_103a, so on this part e4m3 is the only exact
8-bit operand type the fifth-generation tensor cores take.  Compile only: no
GPU is needed and nothing runs."""
import os
import shutil
import subprocess

import pytest

NVCC = os.environ.get("NVCC", shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc")

SRC = r"""
#include <cstdint>
__global__ void k(uint32_t taddr, uint64_t ad, uint64_t bd, uint32_t idesc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}\n"
               :: "r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(1u) : "memory");
}
"""


def _compile(tmp_path, kind, arch):
    src = tmp_path / f"mma_{kind}_{arch}.cu"
    src.write_text(SRC.replace("KIND", kind))
    r = subprocess.run([NVCC, "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", str(src),
                        "-o", str(tmp_path / f"{kind}_{arch}.o")], capture_output=True, text=True)
    return r.returncode, r.stdout + r.stderr


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
def test_kind_i8_is_not_assembled_for_sm_103a(tmp_path):
    rc, out = _compile(tmp_path, "i8", "103a")
    assert rc != 0 and "not supported" in out, out
    rc, out = _compile(tmp_path, "f8f6f4", "103a")
    assert rc == 0, out


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
def test_kind_i8_is_assembled_for_sm_100a(tmp_path):
    rc, out = _compile(tmp_path, "i8", "100a")
    assert rc == 0, out
