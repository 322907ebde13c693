"""Build librom.so (the C-ABI CUDA library) in-tree for sm_103a.

    python -m paper_2009_11742_gb300.build

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``paper_2009_11742_gb300/_build/librom.so``.  Set
``ROM_PTXAS_VERBOSE=1`` to print register / spill / shared-memory use.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librom.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["rom_api.cu", "k_rank2_f32.cu", "k_rank2_f64.cu", "k_rank2_split.cu", "k_rank2_stream.cu", "k_rank2_tc.cu", "k_adjoint.cu", "k_misc.cu",
           "rom_noalloc.cu", "k_stats.cu", "k_fom.cu", "k_peaks.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]
    if os.environ.get("ROM_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def _deps_mtime() -> float:
    newest = 0.0
    for d, _, files in os.walk(CSRC):
        for fn in files:
            if fn.endswith((".cu", ".cuh", ".h")):
                newest = max(newest, os.path.getmtime(os.path.join(d, fn)))
    inc = os.path.join(os.path.dirname(HERE), "include", "rom.h")
    if os.path.exists(inc):
        newest = max(newest, os.path.getmtime(inc))
    return newest


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    nvcc = _nvcc()
    flags = _flags()

    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or os.environ.get("ROM_PTXAS_VERBOSE"):
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
