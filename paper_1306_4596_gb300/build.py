"""Build the sm_103a shared library ``_build/libkfp_swr.so`` with nvcc.

Translation units (``csrc/kfp_swr.cu`` with the host driver and the other kernels,
``csrc/kfp_launch_<precision>_s<shape>.cu`` with the TMA-fed sweep kernels of one
precision and tile shape each, ``csrc/kfp_noalloc.cu`` and ``csrc/kfp_probe.cu``) are
compiled to objects in parallel, one ``-gencode`` (compute_103a / sm_103a), then linked; built in-tree
so that the process loading it is seen using it.  Host code is compiled without
floating-point contraction so that its setup arithmetic (grid nodes, factors)
rounds the same on x86 and Arm.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkfp_swr.so")
SOURCES = [os.path.join(CSRC, f) for f in (
    "kfp_swr.cu", "kfp_noalloc.cu", "kfp_probe.cu",
    # the TMA-fed sweep kernels, one precision and tile shape per translation unit
    "kfp_launch_f64_s0.cu", "kfp_launch_f64_s1.cu", "kfp_launch_f64_s2.cu",
    "kfp_launch_f32_s0.cu", "kfp_launch_f32_s1.cu", "kfp_launch_f32_s2.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(INCLUDE, "kfp_swr.h")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC,-ffp-contract=off",
]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkfp_swr.so")


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if it is missing or older than its sources; return its path."""
    if not force and not is_stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", tag + ".o"))
        cmd = [nvcc(), *NVCC_FLAGS, "-I", INCLUDE, "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    failed = []
    for cmd, proc in procs:
        out, err = proc.communicate()
        if proc.returncode != 0:
            failed.append(f"nvcc failed ({' '.join(cmd)}):\n{out}\n{err}")
        elif verbose:
            print(out, err)
    tmp = LIB + tag + ".so"
    if not failed:
        cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            failed.append(f"link failed ({' '.join(cmd)}):\n{res.stdout}\n{res.stderr}")
    for obj in objs:
        if os.path.exists(obj):
            os.remove(obj)
    if failed:
        raise RuntimeError("\n".join(failed))
    os.replace(tmp, LIB)
    return LIB
