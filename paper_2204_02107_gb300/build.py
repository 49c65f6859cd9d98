"""Builds the in-tree shared library ``libventflow.so`` (CUDA kernels for sm_103a + the C ABI) with nvcc.

The translation units compile in parallel; nothing is installed outside the package directory.  Run as
``python -m paper_2204_02107_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libventflow.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["flow_kernels.cu", "fft_kernels.cu", "fft_reg.cu", "particles.cu", "noalloc.cu", "probe.cu"]
HOST_SOURCES = ["capi.cpp", "batch.cpp", "metrics.cpp"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libventflow.so")


def _compile(args):
    cmd, src = args
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{proc.stdout}\n{proc.stderr}")
    return proc.stderr


def build(verbose=False, extra_flags=()):
    """Compile every source to an object in ``_build/`` and link ``libventflow.so``; returns the library path."""
    nvcc = nvcc_path()
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    objs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", *common, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        jobs.append((cmd, src))
        objs.append(obj)
    for src in HOST_SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        cmd = [nvcc, *common, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, src))
        objs.append(obj)
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_compile, jobs))
    if verbose:
        for log in logs:
            if log:
                sys.stderr.write(log)
    tmp = LIB_PATH + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    proc = subprocess.run(link, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(link)}\n{proc.stdout}\n{proc.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
