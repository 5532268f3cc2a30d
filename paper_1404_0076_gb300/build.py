"""Builds the evaluator's shared library in-tree for GB300 (sm_103a).

    python -m paper_1404_0076_gb300.build

Produces paper_1404_0076_gb300/lib/libinet.so from csrc/ (one CUDA
translation unit and one host C++ unit, compiled in parallel).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libinet.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(INCLUDE, "inet.h"), __file__]
    return all(os.path.getmtime(p) <= t for p in deps)


def build(force: bool = False, verbose: bool = False, extra_nvcc: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    obj_cu = os.path.join(LIBDIR, "inet_api.o")
    obj_cpp = os.path.join(LIBDIR, "inet_text.o")
    nv = nvcc()
    cu = [nv, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "-c", os.path.join(CSRC, "inet_api.cu"), "-o", obj_cu] + (extra_nvcc or [])
    if verbose:
        cu.insert(1, "-Xptxas=-v")
    cpp = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC,
           "-c", os.path.join(CSRC, "inet_text.cpp"), "-o", obj_cpp]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for cmd in (cu, cpp)]
    outs = [p.communicate()[0] for p in procs]
    for p, out, cmd in zip(procs, outs, (cu, cpp)):
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{out}")
        if verbose and out:
            print(out)
    tmp = LIB + ".tmp"
    link = [nv, ARCH, "-shared", "-o", tmp, obj_cu, obj_cpp]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
