"""Build the in-tree CUDA library ``libfsim.so`` for GB300 (sm_103a).

Each translation unit is compiled by nvcc in parallel and the objects are
linked into a shared library next to this file.  The contact kernels are
compiled without FMA contraction so that their float64 distance and
box arithmetic rounds every operation like the CPU reference does.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfsim.so")
# bounds-checked variant (-DFSIM_CHECK): index checks that record and skip
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libfsim_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["capi.cu", "k_local.cu", "k_contact.cu", "k_solve.cu", "k_reduced.cu", "k_pcg.cu",
           "k_schur.cu", "batch.cu", "k_tc.cu", "prefactor.cpp", "serve.cpp", "region.cpp"]
NO_FMA = {"k_contact.cu", "region.cpp"}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _compile(src: str, check: bool = False) -> str:
    obj = os.path.join(BUILD_CHECK if check else BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    flags = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"]
    if check:
        flags += ["-DFSIM_CHECK"]
    if src.endswith(".cu"):
        flags += ARCH + ["--expt-relaxed-constexpr"]
        if src in NO_FMA:
            flags += ["--fmad=false"]
    else:
        flags += ["-x", "c++"]
        if src in NO_FMA:
            flags += ["-Xcompiler", "-ffp-contract=off"]
    cmd = [_nvcc(), "-c", path, "-o", obj] + flags
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "fsim.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile (if sources changed) and return the path of libfsim.so, or of
    the bounds-checked libfsim_check.so with ``check``."""
    lib = LIB_CHECK if check else LIB
    os.makedirs(BUILD_CHECK if check else BUILD, exist_ok=True)
    if not force and not _stale(lib):
        return lib
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda src: _compile(src, check), SOURCES))
    cmd = [_nvcc(), "-shared", "-o", lib] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv)
