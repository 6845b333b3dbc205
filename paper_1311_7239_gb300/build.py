"""Build liblbm.so (the CUDA kernels and the C-ABI of include/lbm.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked with the CUDA runtime into
``paper_1311_7239_gb300/liblbm.so``.  Run ``python -m paper_1311_7239_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "liblbm.so")
DEBUG_LIB = os.path.join(PKG, "liblbm_debug.so")  # -DLBM_DEBUG: kernel index checks (load with LBM_LIBRARY)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile and link liblbm.so (liblbm_debug.so with debug=True: the kernels' index checks);
    returns its path.  Rebuilds only when a source is newer."""
    lib_path = DEBUG_LIB if debug else LIB
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    if debug:
        extra = ("-DLBM_DEBUG", *extra)
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "lbm.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest and not (set(extra) - {"-DLBM_DEBUG"}):
        return lib_path
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {cmd[-3]}")

    with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        list(ex.map(run, cmds))
    tmp = lib_path + ".tmp"
    run([nvcc, *ARCH, "-shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
