"""Builds the in-tree C-ABI library paper_2506_22969_gb300/_build/libsparstencil.so.

CUDA sources are compiled for sm_103a only (``-gencode arch=compute_103a,code=sm_103a``),
host sources with g++; translation units are compiled in parallel and the CUDA runtime is
linked statically.  A content hash of the sources and flags skips rebuilds.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsparstencil.so")
INCLUDE = os.path.join(ROOT, "include")

CU_SOURCES = ["sweep2d.cu", "aux.cu", "noalloc.cu", "correction.cu"]
CPP_SOURCES = ["planner.cpp", "capi.cpp", "server.cpp"]
HEADERS = ["kernels.h", "planner.h", "correction.h"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc() -> str:
    return shutil.which("nvcc") or os.path.join(_cuda_home(), "bin", "nvcc")


ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
if os.environ.get("SPARSTENCIL_DEBUG_TRACE") == "1":  # sweep timeline stamps (debugging only)
    NVCC_FLAGS = NVCC_FLAGS + ["-DSPST_TRACE=1"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function"]


def _digest() -> str:
    h = hashlib.sha256()
    for name in CU_SOURCES + CPP_SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "sparstencil.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + CXX_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links the library if the sources changed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp.txt")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    cuda_inc = os.path.join(_cuda_home(), "include")
    jobs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((src, cmd))
    for src in CPP_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        cmd = [os.environ.get("CXX", "g++"), *CXX_FLAGS, "-I", INCLUDE, "-I", CSRC, "-I", cuda_inc, "-c",
               os.path.join(CSRC, src), "-o", obj]
        jobs.append((src, cmd))
    procs = [(src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for src, cmd in jobs]
    logs = []
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        logs.append(f"== {src}\n{text}")
        if p.returncode != 0:
            failed.append((src, cmd, text))
    with open(os.path.join(BUILD, "build.log"), "w") as f:
        f.write("\n".join(logs))
    if failed:
        src, cmd, text = failed[0]
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{text}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("linking libsparstencil.so failed:\n" + " ".join(link) + "\n" + r.stdout.decode())
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
