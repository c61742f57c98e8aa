"""In-tree build of the native libraries.

- libsp_synth.so  : the seeded input generators (plain C, gcc).
- libsp_gb300.so  : the CUDA Spatial Pooler library behind include/sp.h
                    (nvcc, sm_103a only, -fmad=false so every fp32 step is
                    one round-to-nearest op) and include/sp_loadgen.h (host
                    C++, g++).

Objects are compiled in parallel and cached by modification time under
_build/<arch>/; the shared objects land in _lib/<arch>/.  Both directories are ignored by
git.  Set SP_NVCC_EXTRA for extra nvcc flags.
"""
import concurrent.futures as cf
import os
import platform
import shlex
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
# per-architecture output folders: the same tree is built on x86 and Arm hosts
LIB_DIR = os.path.join(PKG, "_lib", platform.machine())
BUILD_DIR = os.path.join(PKG, "_build", platform.machine())
CSRC = os.path.join(PKG, "csrc")
SYNTH_SRC = os.path.join(PKG, "synth", "synth.c")

SYNTH_LIB = os.path.join(LIB_DIR, "libsp_synth.so")
SP_LIB = os.path.join(LIB_DIR, "libsp_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fvisibility=hidden"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler",
                     "-fPIC,-fvisibility=hidden,-ffp-contract=off", "-DSP_BUILD_LIBRARY",
                     "-I", INCLUDE, "-I", CSRC]


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs


def _newer(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(shlex.quote(c) for c in cmd)
                           + "\n" + r.stdout + r.stderr)
    return r


def build_synth(force=False):
    os.makedirs(LIB_DIR, exist_ok=True)
    if force or _newer(SYNTH_LIB, [SYNTH_SRC, os.path.join(INCLUDE, "sp_synth.h")]):
        tmp = SYNTH_LIB + f".tmp{os.getpid()}"
        _run(["gcc", "-std=c99", "-Wall", "-Wextra"] + CFLAGS + ["-shared", "-o", tmp, SYNTH_SRC])
        os.replace(tmp, SYNTH_LIB)
    return SYNTH_LIB


def cuda_sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def host_sources():
    """Host-only C++ of the library (no device code): built with g++."""
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cpp"))


def build_sp(force=False, jobs=None):
    """Compile every .cu under csrc/ for sm_103a and link libsp_gb300.so."""
    os.makedirs(LIB_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = shlex.split(os.environ.get("SP_NVCC_EXTRA", ""))
    hdrs = _headers()
    jobs_list = []
    objs = []
    for src in cuda_sources():
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _newer(obj, [src] + hdrs):
            jobs_list.append([NVCC] + NVCC_FLAGS + extra + ["-c", src, "-o", obj])
    for src in host_sources():
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _newer(obj, [src] + hdrs):
            jobs_list.append(["g++", "-std=c++17", "-O2", "-fPIC", "-fvisibility=hidden",
                              "-ffp-contract=off", "-Wall", "-DSP_BUILD_LIBRARY", "-I", INCLUDE,
                              "-I", CSRC, "-c", src, "-o", obj])
    synth_obj = os.path.join(BUILD_DIR, "synth.c.o")
    objs.append(synth_obj)
    if force or _newer(synth_obj, [SYNTH_SRC, os.path.join(INCLUDE, "sp_synth.h")]):
        jobs_list.append(["gcc", "-std=c99", "-DSP_SYNTH_HIDDEN"] + CFLAGS
                         + ["-c", SYNTH_SRC, "-o", synth_obj])
    if jobs_list:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 4)) as ex:
            list(ex.map(_run, jobs_list))
    if force or jobs_list or _newer(SP_LIB, objs):
        tmp = SP_LIB + f".tmp{os.getpid()}"
        _run([NVCC] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs
             + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"])
        os.replace(tmp, SP_LIB)
    return SP_LIB


def build_all(force=False):
    return build_synth(force), build_sp(force)


if __name__ == "__main__":
    import sys
    print(build_all(force="--force" in sys.argv))
