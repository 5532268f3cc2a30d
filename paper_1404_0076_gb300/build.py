"""Builds the evaluator's shared library in-tree for GB300 (sm_103a).

    python -m paper_1404_0076_gb300.build

Produces paper_1404_0076_gb300/lib/libinet.so from csrc/ (one CUDA
translation unit and two host C++ units, compiled in parallel).  The device
headers are also embedded in the library (lib/inet_jit_src.inc), which
compiles the rule-specialised asynchronous kernel from them at run time.
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


# Device headers the library embeds for its run-time compile of the
# rule-specialised kernel (NVRTC), in include order.
JIT_HEADERS = [os.path.join(INCLUDE, "inet.h")] + [os.path.join(CSRC, f) for f in
                                                   ("inet_layout.h", "inet_kernels.cuh", "inet_async.cuh")]


def write_jit_sources(path: str) -> None:
    """lib/inet_jit_src.inc: the headers as raw string literals."""
    names, texts = [], []
    for h in JIT_HEADERS:
        text = open(h).read()
        if ')inetsrc"' in text:
            raise RuntimeError(f"{h} holds the raw-string delimiter")
        names.append(os.path.basename(h))
        texts.append(text)
    out = ["// generated by build.py from the device headers; do not edit",
           f"static const int kJitHeaderCount = {len(names)};",
           "static const char* const kJitHeaderNames[] = {" + ", ".join(f'"{n}"' for n in names) + "};",
           "static const char* const kJitHeaderTexts[] = {"]
    out += [f'R"inetsrc({t})inetsrc",' for t in texts]
    out.append("};")
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(out) + "\n")
    os.replace(tmp, path)


def cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "include")


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
    obj_jit = os.path.join(LIBDIR, "inet_jit.o")
    write_jit_sources(os.path.join(LIBDIR, "inet_jit_src.inc"))
    nv = nvcc()
    cu = [nv, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "-c", os.path.join(CSRC, "inet_api.cu"), "-o", obj_cu] + (extra_nvcc or [])
    if verbose:
        cu.insert(1, "-Xptxas=-v")
    cpp = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC,
           "-c", os.path.join(CSRC, "inet_text.cpp"), "-o", obj_cpp]
    jit = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC, "-I", LIBDIR,
           "-I", cuda_include(), "-c", os.path.join(CSRC, "inet_jit.cpp"), "-o", obj_jit]
    cmds = (cu, cpp, jit)
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for cmd in cmds]
    outs = [p.communicate()[0] for p in procs]
    for p, out, cmd in zip(procs, outs, cmds):
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{out}")
        if verbose and out:
            print(out)
    tmp = LIB + ".tmp"
    link = [nv, ARCH, "-shared", "-o", tmp, obj_cu, obj_cpp, obj_jit, "-ldl"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
