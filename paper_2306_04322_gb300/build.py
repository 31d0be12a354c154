"""Build the CUDA library libfs_gb300.so for sm_103a, in-tree.

Every translation unit under csrc/ is compiled by nvcc in parallel, then
linked into one shared library exporting the C ABI of include/fs.h.

build(variant="bounds") builds the bounds-checked library
_build/bounds/libfs_gb300_bounds.so (FS_DEBUG_BOUNDS: every checked global
access outside its buffer sets an error bit and is skipped), the substitute
for a memory checker on small grids; tests load it beside the normal one.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libfs_gb300.so")
VARIANTS = {"release": (BUILD, LIB, []),
            "bounds": (os.path.join(BUILD, "bounds"), os.path.join(BUILD, "bounds", "libfs_gb300_bounds.so"),
                       ["-DFS_DEBUG_BOUNDS"])}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# hidden visibility: only the FS_API entry points of include/fs.h are exported
FLAGS = ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-lineinfo", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=hidden", "-Xcompiler", "-fvisibility-inlines-hidden",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfs_gb300.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), variant: str = "release") -> str:
    out_dir, lib, vflags = VARIANTS[variant]
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    t0 = time.time()
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [cc] + ARCH + FLAGS + vflags + list(extra_flags) + ["-c", src, "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"{os.path.basename(src)}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcuda"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib} in {time.time() - t0:.1f} s")
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          variant="bounds" if "--bounds" in sys.argv else "release")
