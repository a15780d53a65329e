"""Build ``libmlqmc.so`` in-tree with nvcc for sm_103a (no cmake)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmlqmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["mlqmc_cuda.cu", "kl_tcgen05.cu", "rbgs_stream.cu", "rbgs_tma.cu", "resid_tma.cu", "rbgs_whole.cu", "matern_nystrom.cu",
           "mimc.cu", "mlqmc_host.cpp"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-std=c++17", "-O3", "-lineinfo",
           "-Xcompiler", "-fPIC,-ffp-contract=off,-fopenmp", "-I", os.path.join(ROOT, "include")]
    if src.endswith(".cu"):
        cmd += ARCH + ["--expt-relaxed-constexpr"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd += ["-x", "c++"]
    subprocess.check_call(cmd)
    return obj


def build(verbose: bool = False) -> str:
    """Compile every translation unit in parallel and link the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lgomp", "-lcudart", "-lcusolver"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
