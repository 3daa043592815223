"""Build libvup.so in-tree with nvcc for sm_103a (no cmake, parallel units).

``python -m paper_1908_11246_gb300.build`` or ``build()`` compiles every
``csrc/*.cu`` into ``_build/*.o`` and links ``_lib/libvup.so``.  Objects are
rebuilt when their source or any header changed.  ``build(debug=True)`` (or
``--debug``) builds the same units with ``-DVUP_DEBUG`` into
``_build_debug/`` and ``_lib/libvup_debug.so``: device bounds checks that
record an error instead of trapping (the binding loads it when VUP_DEBUG=1).
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
OBJ = os.path.join(PKG, "_build")
OBJ_DEBUG = os.path.join(PKG, "_build_debug")
LIBDIR = os.path.join(PKG, "_lib")
SO = os.path.join(LIBDIR, "libvup.so")
SO_DEBUG = os.path.join(LIBDIR, "libvup_debug.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, verbose: bool, debug: bool = False) -> str:
    obj = os.path.join(OBJ_DEBUG if debug else OBJ, os.path.basename(src)[:-3] + ".o")
    if (os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src)
            and os.path.getmtime(obj) >= _headers_mtime()):
        return obj
    cmd = [NVCC, *ARCH, *FLAGS, *(["-DVUP_DEBUG"] if debug else []), "-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr.strip():
        print(r.stderr, file=sys.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None, debug: bool = False) -> str:
    """Compile all CUDA units and link ``_lib/libvup.so`` (``debug``:
    ``_lib/libvup_debug.so`` with ``-DVUP_DEBUG``); returns its path."""
    so = SO_DEBUG if debug else SO
    os.makedirs(OBJ_DEBUG if debug else OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, debug), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(so) or os.path.getmtime(so) < newest:
        tmp = so + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
