"""Builds the in-tree CUDA library ``_lib/libbiolog.so`` for sm_103a with nvcc.

Two translation units (kernels, host part) compile in parallel and link into
one shared object with the CUDA runtime linked statically. The library is
rebuilt only when a source or header is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libbiolog.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["biolog_kernels.cu", "biolog_host.cpp", "biolog_mlp.cu", "biolog_mlp_host.cpp"]
HEADERS = [os.path.join(CSRC, "biolog_internal.h"), os.path.join(ROOT, "include", "biolog.h")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    tag = f"{os.getpid()}"
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]
    common += os.environ.get("BIOLOG_NVCC_FLAGS", "").split()   # e.g. tuning constants
    objs = [os.path.join(OUT, f"{os.path.splitext(s)[0]}.{tag}.o") for s in SOURCES]
    cmds = []
    for src, obj in zip(SOURCES, objs):
        extra = ARCH + ["-lineinfo"] if src.endswith(".cu") else ["-x", "c++"]
        cmds.append([cc, *common, *extra, "-c", os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(len(cmds)) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
    for c, r in zip(cmds, results):
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(c) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
    tmp = LIB + f".{tag}.tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
