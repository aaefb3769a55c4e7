"""Build the CBC CUDA library in-tree for sm_103a (GB300).

    python -m paper_2601_19650_gb300.build

Every ``csrc/*.cu`` file is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_2601_19650_gb300/libcbc.so`` (the C ABI of ``include/cbc.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcbc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CBC library needs the CUDA toolkit to build")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include"),
                   "--expt-relaxed-constexpr"]


def _compile(src: str, obj: str, extra) -> str:
    cmd = [nvcc()] + _flags() + list(extra) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    return r.stderr


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + [os.path.join(ROOT, "include", "cbc.h")])
    newest_dep = max(os.path.getmtime(d) for d in deps)
    objs, jobs = [], []
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        for s in srcs:
            o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
            objs.append(o)
            if (os.path.exists(o) and os.path.getmtime(o) >= os.path.getmtime(s)
                    and os.path.getmtime(o) >= newest_dep):
                continue
            jobs.append(ex.submit(_compile, s, o, extra))
        for j in jobs:
            msg = j.result()
            if verbose and msg:
                print(msg, file=sys.stderr)
    if (not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
