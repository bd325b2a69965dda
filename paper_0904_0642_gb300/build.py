"""Build libsu3gb300.so in-tree with nvcc for sm_103a (no cmake)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsu3gb300.so")
# the same sources with device bounds checks (SU3_DEBUG_BOUNDS)
BUILD_DBG = os.path.join(HERE, "_build_dbg")
LIB_DBG = os.path.join(HERE, "libsu3gb300_dbg.so")
SOURCES = ["su3_kernels.cu", "su3_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> str:
    """Compile the release library and (debug=True) the debug-bounds library,
    all translation units in parallel; returns the release library's path."""
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "su3.h"))
    targets = [(BUILD, LIB, [])] + ([(BUILD_DBG, LIB_DBG, ["-DSU3_DEBUG_BOUNDS"])] if debug else [])
    jobs, links = [], []
    for bdir, lib, extra in targets:
        os.makedirs(bdir, exist_ok=True)
        objs = []
        compiled = False
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src.replace(".cu", ".o"))
            objs.append(o)
            if force or _stale(o, [s] + headers):
                jobs.append([_nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o])
                compiled = True
        links.append((lib, objs, compiled))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    for lib, objs, compiled in links:
        if force or compiled or _stale(lib, objs):
            run([_nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs, "-lpthread"])
            os.replace(lib + ".tmp", lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
