"""Build the CUDA library in-tree: paper_2112_07537_gb300/_lib/libmrgb.so.

Every translation unit is compiled for sm_103a only, in parallel, then
linked with nvcc into one shared object exporting the C ABI of
include/mrgb.h.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libmrgb.so")
# the ghost kernels: one translation unit per (field type, block type,
# wavelet) instantiation, so that ptxas runs on them in parallel
GHOST_UNITS = [f"ghost_i_{t}{n}{nt}" for t in ("ff", "fd", "dd") for n in (2, 4, 6) for nt in (0, 2)]
# the FP32 stage kernels: one translation unit per wavelet
STAGE_UNITS = [f"stage_i_{n}{nt}" for n in (2, 4, 6) for nt in (0, 2)]
UNITS = ["ghost"] + GHOST_UNITS + STAGE_UNITS + ["boundary", "stencil", "tree", "adapt", "abi", "peaks", "tune"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    hdrs = [os.path.join(SRC, "mr_internal.cuh"), os.path.join(SRC, "ghost_kernels.cuh"),
            os.path.join(SRC, "stage_kernels.cuh"),
            os.path.join(os.path.dirname(HERE), "include", "mrgb.h")]
    nvcc = _nvcc()

    def one(u):
        src = os.path.join(SRC, u + ".cu")
        obj = os.path.join(OUT, u + ".o")
        if force or _stale(obj, [src] + hdrs):
            r = subprocess.run([nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj],
                               capture_output=True, text=True)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {u}.cu:\n{r.stderr}")
            with open(os.path.join(OUT, u + ".ptxas.txt"), "w") as f:
                f.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    if force or _stale(LIB, objs):
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"],
                           capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
