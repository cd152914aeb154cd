"""Builds libcutcell.so (the CUDA path, sm_103a) in-tree with nvcc.

Each translation unit compiles in parallel; geometry.cu is compiled with
-fmad=false so that its FP64 arithmetic is rounded exactly as written.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcutcell.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "cutcell.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "geometry.cu": ["-fmad=false"],
    "step.cu": [],
    "capi.cu": [],
    "noalloc.cu": [],
    "cbcm.cu": [],
    "peak.cu": [],
}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [HEADER, __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")] + ARCH
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *common, *extra, "-c", os.path.join(SRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((unit, out.decode(errors="replace")))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {u}\n{o}" for u, o in failed))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
