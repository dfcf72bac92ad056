"""In-tree build of the CUDA library libdsea.so for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into paper_2507_11289_gb300/_build/libdsea.so (CUDA runtime linked
statically).  Nothing is installed outside the source tree.

build(checked=True) makes the checked variant, _build/libdsea_checked.so,
with -DDSEA_CHECKED=1: every computed global index and shared-memory list
position is tested before use, and one out of range fails the box with
DSEA_ERR_BOUNDS instead of touching memory (a bounds checker for a pool
where compute-sanitizer is not available).  It runs the same arithmetic in
the same order, so its results equal the release build's bit for bit.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdsea.so")
LIB_CHECKED = os.path.join(BUILD, "libdsea_checked.so")
SOURCES = ["dsea_kernels.cu", "dsea_api.cu", "dsea_server.cu", "dsea_noalloc.cu", "dsea_dataset.cu",
           "dsea_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdsea.so")
    return cand


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "dsea.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile (if needed) and return the path of libdsea.so (checked:
    libdsea_checked.so, the bounds-checked variant)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    variant = ["-DDSEA_CHECKED=1"] if checked else []
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-pthread",
              "-I", INCLUDE, "-I", CSRC, *variant, *extra_flags]

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [*common, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread", "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
