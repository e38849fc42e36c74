"""Build the in-tree CUDA library ``libswe.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked with the static
CUDA runtime.  The host mesh builder is compiled without floating-point
contraction so that its geometry is reproducible bit for bit.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libswe.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# Device code is compiled without floating-point contraction (-fmad=false):
# otherwise the compiler (and ptxas, for plain multiplies and adds) may fuse a
# product into a multiply-add differently in each kernel that inlines the same
# function, and the split, tile and batched kernels would round differently.
# Fused multiply-adds that the arithmetic wants are written out (fma_rn).
_V = ["-Xptxas", "-v"] if os.environ.get("SWE_PTXAS_VERBOSE") else []
_NOFMA = ["-fmad=false"]
SOURCES = [
    ("swe_kernels.cu", _NOFMA + _V),
    ("swe_tile.cu", _NOFMA + _V),
    ("swe_noalloc.cu", _NOFMA),
    ("swe_probe.cu", []),
    ("swe_ensemble.cu", _NOFMA + _V),
    ("swe_api.cpp", []),
    ("swe_tiles.cpp", []),
    ("swe_partition.cpp", []),
    ("swe_mesh.cpp", ["-Xcompiler", "-ffp-contract=off"]),
]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h") or f.endswith(".cuh")]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    jobs, objs = [], []
    for src, extra in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(OBJ, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc, "-c", path, "-o", obj, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, *ARCH, *extra]
            jobs.append(cmd)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        return p.stdout + p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for out in ex.map(run, jobs):
            if verbose and out:
                print(out, file=sys.stderr)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, "-shared", *ARCH, "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
