"""Builds libgbdgemm.so in-tree from csrc/*.cu with nvcc for sm_103a only.

Every translation unit is compiled in parallel; the shared library is linked
with the static CUDA runtime.  Nothing here needs a GPU (nvcc cross-compiles).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgbdgemm.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
          "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps()) and os.path.getmtime(__file__) <= t


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC] + ARCH + CFLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile (if stale) and return the path of libgbdgemm.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    srcs = _sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


CPU_SRC = os.path.join(PKG, "cpu", "gbd_cpu.c")
CPU_LIB = os.path.join(PKG, "libgbdcpu.so")
CC = os.environ.get("CC", "gcc")


def build_cpu(force: bool = False) -> str:
    """Compile (if stale) and return the path of libgbdcpu.so, the host DGEMM of the paper's
    five loops (portable C: no target-specific flags, so x86-64 and aarch64 builds agree)."""
    deps = [CPU_SRC, os.path.join(INCLUDE, "gbdcpu.h"), __file__]
    if not force and os.path.exists(CPU_LIB) and all(os.path.getmtime(d) <= os.path.getmtime(CPU_LIB) for d in deps):
        return CPU_LIB
    tmp = CPU_LIB + f".tmp{os.getpid()}"
    cmd = [CC, "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fvisibility=hidden", "-I" + INCLUDE,
           "-o", tmp, CPU_SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"{CC} failed on gbd_cpu.c:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, CPU_LIB)
    return CPU_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
    print(build_cpu(force="--force" in sys.argv))
