"""Build libfe.so (CUDA sources for sm_103a) in-tree under _lib/."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
SO = os.path.join(LIBDIR, "libfe.so")
# the FE_DEBUG_BOUNDS build: kernels check their indirect indices (see fe_idx)
SO_DEBUG = os.path.join(LIBDIR, "dbg", "libfe_dbg.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["fe_mesh.cu", "fe_assemble.cu", "fe_krylov.cu", "nl_solve.cu", "fe_amg.cu", "fe_noalloc.cu", "fe_serve.cu",
           "fe_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.extend(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(so=SO):
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False, debug_bounds=False):
    """Compile libfe.so (or, debug_bounds=True, the index-checking
    libfe_dbg.so with -DFE_DEBUG_BOUNDS) in-tree for sm_103a."""
    so = SO_DEBUG if debug_bounds else SO
    if not force and up_to_date(so):
        return so
    objdir = os.path.dirname(so)
    os.makedirs(objdir, exist_ok=True)
    extra = ["-DFE_DEBUG_BOUNDS"] if debug_bounds else []

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    tmp = so + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    import sys
    build(force=True, verbose="-v" in sys.argv)
    print(SO)
