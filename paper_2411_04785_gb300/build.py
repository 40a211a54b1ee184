"""Build libcompton.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled to an object in parallel, then linked into a shared
library next to this file.  No cmake; a full rebuild takes well under a
minute.  ``python -m paper_2411_04785_gb300.build`` runs it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcompton.so")
# The debug build: every checked index is compared with its buffer's bound and
# a failure is recorded in one device word instead of being accessed
# (cc_debug_bounds); relocatable device code lets every translation unit reach
# that word.
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libcompton_debug.so")
DEBUG_FLAGS = ["-DCC_DEBUG_BOUNDS", "-rdc=true"]
SOURCES = ["capi.cu", "recon.cu", "sweep.cu", "refine.cu", "grid.cu", "trace.cu", "cluster.cu", "voxel.cu",
           "noalloc.cu", "mlp.cu", "selftest.cu", "order.cu"]
INCLUDE = os.path.join(HERE, "..", "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xptxas", "-v", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcompton.so")
    return p


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


_INCLUDE_RE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def _deps(path: str, seen=None) -> set:
    """The file and every header it includes with quotes, transitively (found
    next to the including file or in include/), so that editing any of them
    rebuilds the objects that use it."""
    seen = set() if seen is None else seen
    if path in seen:
        return seen
    seen.add(path)
    with open(path) as f:
        text = f.read()
    for name in _INCLUDE_RE.findall(text):
        for d in (os.path.dirname(path), INCLUDE):
            cand = os.path.normpath(os.path.join(d, name))
            if os.path.exists(cand):
                _deps(cand, seen)
                break
    return seen


def _compile(src: str, verbose: bool, debug: bool = False) -> str:
    obj = os.path.join(BUILD_DEBUG if debug else BUILD, os.path.splitext(src)[0] + ".o")
    deps = sorted(_deps(os.path.join(CSRC, src)))
    if os.path.exists(obj) and os.path.getmtime(obj) >= _newest(deps):
        return obj
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *(DEBUG_FLAGS if debug else []), "-c",
           os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    with open(obj + ".ptxas.txt", "w") as f:   # -Xptxas -v report
        f.write(r.stderr)
    if verbose:
        print(f"[build] {src}", file=sys.stderr)
    return obj


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    """Compile and link libcompton.so (debug=True: libcompton_debug.so, the
    build with index bounds checks); returns its path."""
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    if force:
        for f in os.listdir(bdir):
            os.remove(os.path.join(bdir, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, debug), SOURCES))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < _newest(objs):
        tmp = lib + f".tmp{os.getpid()}"
        link_objs = list(objs)
        if debug:      # device link of the relocatable objects
            dlink = os.path.join(bdir, "dlink.o")
            r = subprocess.run([_nvcc(), *ARCH, "-dlink", "-Xcompiler", "-fPIC", *objs,
                                "-o", dlink], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"device link failed:\n{r.stdout}\n{r.stderr}")
            link_objs.append(dlink)
        cmd = [_nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *link_objs, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, debug="--debug" in sys.argv))
