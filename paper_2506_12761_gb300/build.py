"""Build the two libraries in-tree.

libvelopir.so (the GPU library, velopir.h): every CUDA translation unit
compiles for sm_103a (GB300) with nvcc in parallel, then nvcc links it.
libvelopir_client.so (the host-only client library, velopir_client.h): one
C++ file compiled with the host compiler, linked against no CUDA library.
Outputs sit beside this file (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvelopir.so")
CLIENT_LIB = os.path.join(HERE, "libvelopir_client.so")
CLIENT_SOURCE = "client.cpp"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "br_dense.cu", "br_ntt.cu", "br_tc.cu", "keyswitch.cu", "sched.cpp", "plan.cpp", "noalloc.cu", "client_gpu.cu"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvelopir.so")


def _compile(src: str, verbose_ptxas: bool) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
           "-I", os.path.join(HERE, "..", "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose_ptxas and src.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def _fresh(out: str, deps) -> bool:
    return os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in deps)


def build_client(force: bool = False) -> str:
    """libvelopir_client.so with the host C++ compiler (no CUDA)."""
    inc = os.path.join(HERE, "..", "include")
    deps = [os.path.join(CSRC, CLIENT_SOURCE), os.path.join(inc, "velopir_client.h"), os.path.join(inc, "velopir_common.h")]
    if not force and _fresh(CLIENT_LIB, deps):
        return CLIENT_LIB
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("no host C++ compiler found for libvelopir_client.so")
    tmp = CLIENT_LIB + ".tmp%d" % os.getpid()
    cmd = [cxx, "-std=c++17", "-O3", "-fPIC", "-shared", "-pthread", "-Wall", "-I", inc, deps[0], "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed on {CLIENT_SOURCE}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, CLIENT_LIB)
    return CLIENT_LIB


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Both libraries; returns the GPU library's path."""
    with cf.ThreadPoolExecutor(1) as ex:
        client = ex.submit(build_client, force)
        lib = _build_gpu(force, verbose_ptxas)
        client.result()
    return lib


def _build_gpu(force: bool, verbose_ptxas: bool) -> str:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")]
    deps += [os.path.join(HERE, "..", "include", h) for h in ("velopir.h", "velopir_common.h")]
    if not force and _fresh(LIB, deps):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
    print(CLIENT_LIB)
