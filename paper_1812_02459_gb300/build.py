"""Build the CUDA library liblbm.so (sm_103a) in-tree with nvcc.

The library is the product: every step of the lattice update runs in its
kernels.  It is compiled for sm_103a only (``-gencode
arch=compute_103a,code=sm_103a``), with the CUDA runtime linked statically.
Beside it, liblbm_debug.so is the same source built with LBM_DEBUG, whose
FP32 kernels check their paired shared-memory accesses against the launch's
dynamic shared memory (lbm_debug_violations reports the first miss); the
two are compiled at the same time.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbm.so")
DEBUG_LIB = os.path.join(HERE, "liblbm_debug.so")
SOURCES = [os.path.join(CSRC, n) for n in ("lbm_api.cu", "lbm_noalloc.cu", "lbm_adjoint.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "lbm_kernels.cuh"), os.path.join(CSRC, "lbm_internal.h"),
                  os.path.join(CSRC, "lbm_jit.h"), os.path.join(INCLUDE, "lbm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")
    return cand


def _stale(lib):
    return not os.path.exists(lib) or any(os.path.getmtime(d) > os.path.getmtime(lib) for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liblbm.so and liblbm_debug.so if missing or older than any
    source (both at once); return the path of liblbm.so."""
    jobs = []
    for lib, extra in ((LIB, []), (DEBUG_LIB, ["-DLBM_DEBUG"])):
        if not force and not _stale(lib):
            continue
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", *extra,
               "-I", INCLUDE, "-o", tmp, *SOURCES, "-ldl"]
        if verbose and not extra:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((lib, tmp, subprocess.Popen(cmd)))
    failed = [lib for lib, tmp, proc in jobs if proc.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, f"nvcc ({', '.join(os.path.basename(f) for f in failed)})")
    for lib, tmp, _ in jobs:
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
