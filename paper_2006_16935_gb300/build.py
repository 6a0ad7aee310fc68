"""Builds libqfd.so (the CUDA kernels and the C ABI of include/qfd.h) in-tree for sm_103a.

qfd_inst.cu is compiled once per (arithmetic policy, lattice size) pair and
every object by its own nvcc process in parallel; the objects are linked into
paper_2006_16935_gb300/libqfd.so with the CUDA runtime linked statically.
Rebuilds only when a source is newer than the library.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqfd.so")
POLICIES = ["DF", "F64", "F32"]  # slowest first
SIZES = [1024, 512, 256, 192, 128, 96, 64, 32, 16, 8]
UNITS = ([("qfd_inst.cu", f"inst_{p}_{n}", ["-DQFD_POLICY=" + p, f"-DQFD_N={n}"]) for p in POLICIES for n in SIZES]
         + [("qfd_api.cu", "api", []), ("qfd_noalloc.cu", "noalloc", []), ("qfd_peaks.cu", "peaks", [])])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "qfd.h"))
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build_library(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, name, defs = unit
        obj = os.path.join(BUILD, name + ".o")
        cmd = [nvcc, *FLAGS, *ARCH, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    workers = max(2, min(len(UNITS), os.cpu_count() or 4))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
