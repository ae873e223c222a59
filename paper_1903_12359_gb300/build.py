"""Build the CUDA library libpgcp.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel into _build/ and linked
into paper_1903_12359_gb300/libpgcp.so.  The welding unit is compiled without
FMA contraction so its FP64 arithmetic rounds exactly like the CPU reference.
Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpgcp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["primitives.cu", "partition.cu", "schedule.cu", "assemble.cu", "pcg.cu", "pcg_df.cu", "pcg_ml.cu", "weld.cu",
           "solve.cu", "qcfix.cu", "metrics.cu", "area.cu", "gemm_tc.cu", "mpnn.cu", "api.cu"]
NO_FMA = {"weld.cu"}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(src: str) -> list:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "-I" + os.path.join(ROOT, "include")]
    if src in NO_FMA:
        f += ["-fmad=false"]
    return f


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, "pgcp_internal.h"),
                                                         os.path.join(CSRC, "df_arith.cuh"),
                                                         os.path.join(ROOT, "include", "pgcp.h"),
                                                         os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
