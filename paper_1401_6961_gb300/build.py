"""Builds the CUDA library ``_build/libkx.so`` for sm_103a with nvcc.

Every translation unit is compiled in parallel (one process each) and
relinked only when a source or header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
OBJ = os.path.join(OUT, "obj")
LIB = os.path.join(OUT, "libkx.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkx")
    return exe


def sources():
    return sorted(glob.glob(os.path.join(SRC, "*.cu")))


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-4000:]}")
    os.replace(obj + ".tmp", obj)
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def _weight(src: str) -> int:
    """Rough compile cost of a translation unit: the per-bra-class ERI units
    grow with the bra's angular momentum (the double-word ones stop at
    la+lb+lc+ld = 5, so their heaviest bras are the middle ones)."""
    b = os.path.basename(src)
    for pre, base in (("kx_eri_dw_", 2), ("kx_eri_", 4)):
        if b.startswith(pre) and b[len(pre):len(pre) + 2].isdigit():
            la, lb = int(b[len(pre)]), int(b[len(pre) + 1])
            return base + (la + lb if pre == "kx_eri_" else min(la + lb, 5 - la - lb) + 1)
    return 6 if b.startswith("kx_eri_big") else 0


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile (if needed) and link libkx.so; returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    srcs = sources()
    hdr = _headers_mtime()
    todo = []
    for s in srcs:
        obj = os.path.join(OBJ, os.path.basename(s)[:-3] + ".o")
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(s), hdr):
            todo.append(s)
    if todo:
        # heaviest translation units first
        todo.sort(key=lambda s: -_weight(s))
        n = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(n) as ex:
            list(ex.map(lambda s: _compile(s, verbose), todo))
    objs = [os.path.join(OBJ, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
