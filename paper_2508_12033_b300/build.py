"""Build step: compile the CUDA library in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liblrdmc.so")
# the checked build: data-derived indices tested in the kernels (LRDMC_CHECKED)
LIB_CHECKED = os.path.join(PKG, "liblrdmc_checked.so")
ARCH = "arch=compute_103a,code=sm_103a"


def _sources():
    out = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))]
    out.append(os.path.join(INCLUDE, "lrdmc.h"))
    return out


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    p = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(p):
        return p
    raise RuntimeError("nvcc not found")


def nvcc_command(out: str = LIB, extra=()):
    return [nvcc_path(), "-std=c++17", "-O3", "-gencode", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
            "-shared", "-I", INCLUDE, *extra, "-o", out, os.path.join(CSRC, "lrdmc.cu")]


def is_stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile liblrdmc.so (and, with checked, liblrdmc_checked.so) next to
    this file if missing or older than a source."""
    targets = [(LIB, ())] + ([(LIB_CHECKED, ("-DLRDMC_CHECKED",))] if checked else [])
    for lib, extra in targets:
        if force or is_stale(lib):
            tmp = f"{lib}.{os.getpid()}.tmp"   # per process: concurrent builds never share a file
            cmd = nvcc_command(tmp, extra)
            if verbose:
                print(" ".join(cmd))
            subprocess.run(cmd, check=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
