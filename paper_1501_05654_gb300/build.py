"""Builds librsg.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
library exporting the C ABI of include/rsg.h.  No cmake, portable host flags
only (the library is rebuilt on x86 and on Arm hosts).
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librsg.so")
# (source, extra flags): the stencil kernels are compiled once per precision,
# the complex64 row-TMA kernels separately (parallel compiles)
SOURCES = [("rsg_kernels.cu", ["-DRSG_ONLY_FLOAT"]), ("rsg_kernels.cu", ["-DRSG_ONLY_FLOAT", "-DRSG_ROWTMA_TU"]),
           ("rsg_kernels.cu", ["-DRSG_ONLY_DOUBLE"]),
           ("rsg_quad.cu", []), ("rsg_wide.cu", []), ("rsg_bstep.cu", []), ("rsg_scaled.cu", []), ("rsg_selftest.cu", []), ("rsg_linalg.cu", []), ("rsg_noalloc.cu", []), ("rsg_host.cpp", [])]
HEADERS = ["rsg_internal.h", "rsg_vec.cuh", "rsg_async.cuh", "rsg_batch.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librsg.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in sorted({s for s, _ in SOURCES}) + HEADERS]
    deps.append(os.path.join(ROOT, "include", "rsg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include")]
    if ptxas_info:
        common += ["-Xptxas", "-v"]

    def one(item):
        i, (src, flags) = item
        obj = os.path.join(OUT, f"{src}.{i}.{os.getpid()}.o")
        cmd = [cc] + common + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, enumerate(SOURCES)))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
