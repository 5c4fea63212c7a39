"""Build step for libcoop.so (nvcc, sm_103a only).

``build_library()`` compiles ``csrc/coop.cu`` into ``libcoop.so`` inside the package
directory (in-tree, git-ignored).  It is what the repository's ``build()`` calls and
what the binding calls when the library is missing or older than its sources.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(PKG, "libcoop.so")
SOURCES = [os.path.join(PKG, "csrc", "coop.cu")]
HEADERS = glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + [
    os.path.join(os.path.dirname(PKG), "include", "coop.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcoop.so")
    return cand


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS if os.path.exists(s))


def build_command(out: str) -> list:
    # -rdc + cudadevrt: the kernels launch their own forked CTAs (device-side launches)
    return [nvcc_path(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-rdc=true", "-shared", "-Xcompiler", "-fPIC",
            "-o", out, *SOURCES, "-lcudadevrt"]


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile libcoop.so if it is missing or stale; returns its path."""
    if force or needs_build():
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = build_command(tmp)
        res = subprocess.run(cmd, capture_output=not verbose, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + (res.stderr or "") + (res.stdout or ""))
        os.replace(tmp, LIB)
    return LIB
