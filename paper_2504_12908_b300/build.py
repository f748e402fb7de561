"""Builds the in-tree C-ABI library libipc_b300.so for sm_103a with nvcc.

Usage: python -m paper_2504_12908_b300.build  (or build() from Python).
Objects are compiled in parallel into _build/ beside this file and linked
into paper_2504_12908_b300/libipc_b300.so.  build(checks=True) (or
--checks) builds the bounds-checked variant libipc_b300_checks.so
(-DIPC_CHECKS: the kernels test the indices they gather through and record
the first violation instead of making the access; see ipc_check_report).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libipc_b300.so")
BUILD = os.path.join(HERE, "_build")
OUT_CHECKS = os.path.join(HERE, "libipc_b300_checks.so")
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
SOURCES = ["scene.cpp", "kernels_contact.cu", "kernels_solver.cu", "kernels_pcg.cu", "capi.cu", "noalloc.cu",
           "tactile.cu", "peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                     "-Xptxas", "-O3", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _compile(src: str, verbose_ptxas: bool, checks: bool = False) -> str:
    obj = os.path.join(BUILD_CHECKS if checks else BUILD, os.path.splitext(src)[0] + ".o")
    flags = list(NVCC_FLAGS) + (["-DIPC_CHECKS"] if checks else [])
    if verbose_ptxas and src.endswith(".cu"):
        flags += ["-Xptxas", "-v"]
    cmd = [_nvcc()] + flags + ["-x", "cu" if src.endswith(".cu") else "c++", "-c",
                               os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-c",
               os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    for root in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(root):
            if os.path.getmtime(os.path.join(root, f)) > t:
                return True
    return False


def build(force: bool = False, verbose_ptxas: bool = False, checks: bool = False) -> str:
    """Compile and link the library (or its bounds-checked variant) if any
    source is newer; returns its path."""
    out = OUT_CHECKS if checks else OUT
    if not force and not _stale(out):
        return out
    os.makedirs(BUILD_CHECKS if checks else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, checks), SOURCES))
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", out] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checks="--checks" in sys.argv))
