"""Build the CUDA library librewl.so (sm_103a) in-tree.

The translation units are compiled in parallel with nvcc and linked into
paper_1312_3004_gb300/_build/librewl.so.  No CPU code path is built: the
library is the GPU implementation only.  build(debug=True) builds
librewl_debug.so instead, with the kernels' bounds checks compiled in
(REWL_DEBUG_CHECKS: an out-of-range index is recorded and replaced, and the
run returns REWL_ERR_STATE); the package loads it when REWL_DEBUG=1.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librewl.so")
LIB_DEBUG = os.path.join(OUT_DIR, "librewl_debug.so")
SOURCES = ["rewl_kernels.cu", "rewl_sweep.cu", "rewl_host.cu", "rewl_batch.cu", "rewl_server.cu", "rewl_static.cu",
           "rewl_analysis.cu", "rewl_probe.cu", "rewl_production.cu"]
HEADERS = ["rewl_internal.cuh", "rewl_host_internal.hpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _cuda_lib_dir():
    return os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps += [os.path.join(ROOT, "include", "rewl.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in deps):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if debug:
        common.append("-DREWL_DEBUG_CHECKS")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src + (".debug.o" if debug else ".o"))
        objs.append(obj)
        cmd = [nvcc, "-c"] + common + ["-o", obj, os.path.join(CSRC, src)]
        if verbose:
            cmd.insert(2, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd)))
    for cmd, p in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = lib + ".tmp.%d" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath," + _cuda_lib_dir()]
    subprocess.run(link, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
