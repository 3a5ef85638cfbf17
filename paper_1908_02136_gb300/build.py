"""Build libkpp.so in-tree with nvcc for sm_103a (GB300).

Every ``csrc/*.cu`` is compiled to an object in parallel and linked into
``paper_1908_02136_gb300/_build/libkpp.so``; the debug build (``KPP_DEBUG=1``:
index checks before the hot kernels' memory accesses, reported as a device
status) goes to ``_build_debug/libkpp.so``.  Rebuilds only when a source or
header is newer than the library.  No cmake, no torch extension machinery.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libkpp.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libkpp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe


def _flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
            "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC, *extra]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def lib_path(debug: bool = False) -> str:
    return LIB_DEBUG if debug else LIB


def stale(debug: bool = False) -> bool:
    lib = lib_path(debug)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _compile_jobs(debug: bool, extra):
    out = BUILD_DEBUG if debug else BUILD
    flags = _flags(list(extra) + (["-DKPP_DEBUG=1"] if debug else []))
    return [(src, os.path.join(out, os.path.basename(src)[:-3] + ".o"), flags)
            for src in sources()]


def _link(objs, lib):
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          debug: bool = True) -> str:
    """Compile and link libkpp.so (and, with ``debug``, its KPP_DEBUG build,
    compiled in the same parallel pool); returns the release library's path."""
    variants = [False] + ([True] if debug else [])
    todo = [v for v in variants if force or stale(v)]
    if not todo:
        return LIB
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    jobs = []
    for v in todo:
        os.makedirs(BUILD_DEBUG if v else BUILD, exist_ok=True)
        jobs += [(v, *j) for j in _compile_jobs(v, extra)]

    def compile_one(job):
        _, src, obj, flags = job
        cmd = [nvcc(), "-c", src, "-o", obj, *flags]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for v in todo:
        _link([o for j, o in zip(jobs, objs) if j[0] == v], lib_path(v))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
