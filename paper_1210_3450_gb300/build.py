"""Build the CUDA library ``_build/libljmd.so`` for sm_103a with nvcc.

Translation units are compiled in parallel, then linked into one shared
library that exports the C ABI of ``include/ljmd.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libljmd.so")
SOURCES = ["ljmd_kernels.cu", "ljmd_engine.cu", "ljmd_capi.cu", "ljmd_noalloc.cu", "ljmd_bubbles.cu",
           "ljmd_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-fvisibility=hidden", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libljmd")
    return cand


def _deps() -> list[str]:
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "ljmd.h"))
    return out


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link if any source is newer than the library; return its path.
    checked=True builds the variant with device bounds checks (LJMD_CHECKS) into
    _build/checked/libljmd.so."""
    out_dir = os.path.join(OUT_DIR, "checked") if checked else OUT_DIR
    lib = os.path.join(out_dir, "libljmd.so")
    flags = NVCC_FLAGS + (["-DLJMD_CHECKS"] if checked else [])
    os.makedirs(out_dir, exist_ok=True)
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(p) for p in _deps())
        if os.path.getmtime(lib) >= newest:
            return lib
    nvcc = _nvcc()
    objs = []

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """The product library and the checked variant, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, verbose, c) for c in (False, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv, verbose=True))
