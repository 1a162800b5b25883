"""Build libkm.so (the C ABI over the sm_103a kernels) in-tree with nvcc.

Each .cu file is compiled to an object in parallel, then linked into
``paper_2405_12052_gb300/libkm.so``.  Only sm_103a code is generated.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libkm.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["km_assign.cu", "km_assign_tc.cu", "km_update.cu", "km_api.cu", "km_noalloc.cu", "km_gemm.cu", "km_msort.cu",
           "km_batch.cu", "km_batch_api.cu", "km_kpp.cu",
           "km_setnet.cu", "km_setnet_api.cu", "km_objective.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "km.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        log = os.path.join(BUILD, src.replace(".cu", ".log"))
        extra = os.environ.get("KM_NVCC_EXTRA", "").split()
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, obj, log, subprocess.Popen(cmd, stdout=open(log, "w"), stderr=subprocess.STDOUT)))
    objs = []
    for src, obj, log, p in procs:
        if p.wait() != 0:
            sys.stderr.write(open(log).read())
            raise RuntimeError(f"nvcc failed on {src}")
        if verbose:
            sys.stderr.write(open(log).read())
        objs.append(obj)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
