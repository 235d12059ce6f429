"""Builds the CUDA library (libpagd.so, sm_103a) in-tree.

``build_library()`` compiles ``csrc/pagd.cu`` with nvcc for
``-gencode arch=compute_103a,code=sm_103a``.  ``build_emulation()`` compiles the
same source as host C++ with ``-DPAGD_EMU`` into ``libpagd_emu.so``: a test
harness that runs the kernel's phases block by block on the CPU so that index
arithmetic and control flow can be checked without a GPU.  The product binding
never loads the emulation library.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpagd.so")
EMU = os.path.join(BUILD, "libpagd_emu.so")
# host code, one kernel translation unit per fixed line length (0: runtime length)
# the batched kernel per iteration precision, and the learned-guess network
SOURCES = (["pagd.cu"] + [f"pagd_k{nf}_{t}.cu" for nf in (0, 64, 128, 256, 512) for t in ("f32", "f64")]
           + ["pagd_batch_f32.cu", "pagd_batch_f64.cu", "sno.cu"])
HEADERS = ["compat.cuh", "fft.cuh", "solver.cuh", "cluster.cuh", "kernels.cuh", "batch.cuh"]
GENCODE = "arch=compute_103a,code=sm_103a"


def _deps():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(os.path.dirname(HERE), "include", "pagd.h"))
    files.append(os.path.join(os.path.dirname(HERE), "include", "pagd_sno.h"))
    return files


def _stale(target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(f) > t for f in _deps())


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpagd.so")
    return path


def build_library(force: bool = False, verbose: bool = False) -> str:
    """nvcc each translation unit for sm_103a in parallel, then link the .so."""
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale(LIB):
        return LIB
    tag = os.getpid()
    flags = ["-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
    if verbose:
        flags.append("-Xptxas=-v")

    def compile_one(src):
        obj = os.path.join(BUILD, f"{os.path.splitext(src)[0]}.{tag}.o")
        subprocess.check_call([nvcc(), *flags, "-c", "-o", obj, os.path.join(CSRC, src)])
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{tag}.tmp"
    subprocess.check_call([nvcc(), "-gencode", GENCODE, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


def build_emulation(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not _stale(EMU):
        return EMU
    tmp = EMU + f".{os.getpid()}.tmp"
    cxx = shutil.which("g++") or "g++"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-DPAGD_EMU", "-x", "c++", "-fPIC", "-shared",
                           "-o", tmp, os.path.join(CSRC, "pagd.cu")])
    os.replace(tmp, EMU)
    return EMU
