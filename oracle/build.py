"""Build the CPU oracle (test infrastructure only) into oracle/_lib/<arch>/.

The oracle is plain C++ compiled with -O2 -ffp-contract=off (no FMA
contraction, no fast-math) so that its fp32 steps round exactly as written.
"""
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(HERE, "_lib", platform.machine())
LIB_PATH = os.path.join(LIB_DIR, "libsp_oracle.so")
SOURCES = [os.path.join(HERE, "sp_oracle.cpp")]
HEADERS = [os.path.join(HERE, "sp_oracle.h")]


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in SOURCES + HEADERS)


def build(force: bool = False) -> str:
    if force or _stale():
        os.makedirs(LIB_DIR, exist_ok=True)
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-Wextra", "-fPIC", "-shared", "-o", tmp] + SOURCES
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True))
