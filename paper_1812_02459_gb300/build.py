"""Build the CUDA library liblbm.so (sm_103a) in-tree with nvcc.

The library is the product: every step of the lattice update runs in its
kernels.  It is compiled for sm_103a only (``-gencode
arch=compute_103a,code=sm_103a``), with the CUDA runtime linked statically.
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
SOURCES = [os.path.join(CSRC, n) for n in ("lbm_api.cu", "lbm_noalloc.cu", "lbm_adjoint.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "lbm_kernels.cuh"), os.path.join(CSRC, "lbm_internal.h"),
                  os.path.join(CSRC, "lbm_jit.h"), os.path.join(INCLUDE, "lbm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")
    return cand


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liblbm.so if missing or older than any source; return its path."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", INCLUDE, "-o", tmp, *SOURCES, "-ldl"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
