"""Builds libofm.so (the C-ABI library) in-tree for sm_103a.

nvcc compiles each CUDA translation unit with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` in parallel, g++
compiles the host-only planner, and nvcc links a shared library with the
CUDA runtime linked statically.  Objects go to ``_build/`` next to this file;
a unit is rebuilt when it or any header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libofm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the OFM library needs the CUDA toolkit to build")


def _cuda_include(nvcc):
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    hs.append(os.path.join(INCLUDE, "ofm.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src, nvcc, verbose, extra):
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    inc = ["-I", INCLUDE, "-I", CSRC]
    if src.endswith(".cu"):
        cmd = [nvcc, "-c", path, "-o", obj] + ARCH + NVCC_FLAGS + inc + extra
    else:
        cxx = os.environ.get("CXX", "g++")
        cmd = [cxx, "-c", path, "-o", obj] + CXX_FLAGS + inc + ["-I", _cuda_include(nvcc)]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          ptxas_verbose: bool = False) -> str:
    """Compile (if needed) and link libofm.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "MACHINE")
    machine = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != machine:
        force = True          # objects from another architecture are never reused
    hmt = _headers_mtime()
    todo, objs = [], []
    for s in sources():
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(
                os.path.getmtime(os.path.join(CSRC, s)), hmt):
            todo.append(s)
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    logs = {}
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(8, len(todo))) as ex:
            futs = {ex.submit(_compile, s, nvcc, verbose, extra): s for s in todo}
            for f in cf.as_completed(futs):
                _, log = f.result()
                logs[futs[f]] = log
    if (todo or force or not os.path.exists(LIB)
            or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs)):
        tmp = LIB + ".tmp"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"linking libofm.so failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(machine + "\n")
    if ptxas_verbose:
        for s, log in sorted(logs.items()):
            print(f"== {s}\n{log}")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                ptxas_verbose="--ptxas" in sys.argv))
