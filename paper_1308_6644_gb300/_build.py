"""Build the in-tree CUDA library ``libnuasm.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel to an object file under
``_build/`` and the objects are linked into ``paper_1308_6644_gb300/libnuasm.so``.
A rebuild happens only when a source or header is newer than the library.
No CMake; host code is portable C++ (the library is built on x86-64 and on
aarch64 hosts alike).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libnuasm.so")

SOURCES = ["capi.cu", "resources.cu", "passes.cu", "passes_row_f32.cu", "passes_col_f32.cu", "passes_row_f64.cu",
           "passes_col_f64.cu", "gridding.cu", "hostmath.cpp", "noalloc.cu", "rs.cu", "batch.cu", "serve.cu", "diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnuasm.so")


def _deps() -> list[str]:
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".cpp", ".h")):
                out.append(os.path.join(d, f))
    return out


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(nvcc: str, src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link libnuasm.so; returns its path."""
    if not force and not needs_build():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


DEBUG_LIB = os.path.join(PKG, "libnuasm_debug.so")


def build_debug(force: bool = False) -> str:
    """Compile the bounds-checking debug library ``libnuasm_debug.so`` (every
    translation unit with NUASM_DEBUG_BOUNDS=1, objects under _build/debug);
    returns its path.  Selected at run time with NUASM_LIBRARY."""
    if not force and os.path.exists(DEBUG_LIB) and \
            not any(os.path.getmtime(f) > os.path.getmtime(DEBUG_LIB) for f in _deps()):
        return DEBUG_LIB
    nvcc = _nvcc()
    bdir = os.path.join(BUILD, "debug")
    os.makedirs(bdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, ["-DNUASM_DEBUG_BOUNDS=1"], bdir), SOURCES))
    tmp = DEBUG_LIB + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, DEBUG_LIB)
    return DEBUG_LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
