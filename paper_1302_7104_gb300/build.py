"""Build the CUDA library ``libpclb.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into a shared
library inside the package (``paper_1302_7104_gb300/_build/``).  Rebuilds only
when a source or header is newer than the library.  The benchmark's
measurement helper (``csrc/bench/``) is linked into a library of its own,
``libpclb_bench.so``, which the product never loads.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libpclb.so")
BENCH_SRC = os.path.join(CSRC, "bench")
BENCH_LIB = os.path.join(OUT, "libpclb_bench.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
         "-Xptxas", "-warn-spills"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def _bench_sources():
    return sorted(glob.glob(os.path.join(BENCH_SRC, "*.cu")))


def stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(BENCH_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(BENCH_LIB))
    return any(os.path.getmtime(p) > t for p in _deps() + _bench_sources())


def _compile(src: str, verbose: bool) -> str:
    tag = "bench_" if os.path.dirname(src) == BENCH_SRC else ""
    obj = os.path.join(OUT, tag + os.path.basename(src) + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libpclb.so; returns its path."""
    if not force and not stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    srcs, bsrcs = _sources(), _bench_sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs + bsrcs))
    _link(LIB, objs[:len(srcs)])
    _link(BENCH_LIB, objs[len(srcs):])
    return LIB


def _link(lib: str, objs) -> None:
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc link failed for {os.path.basename(lib)}:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
