"""Builds libpkmom.so in-tree for sm_103a with nvcc (one object per .cu, in parallel),
and its checked variant libpkmom_checked.so (-DPKMOM_CHECKED=1: index tests before
every grid, buffer and bin access).

Usage: python -m paper_2005_06170_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpkmom.so")
OUT_DIR_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libpkmom_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libpkmom")
    return exe


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
        [os.path.join(ROOT, "include", "pkmom.h")]


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """Both libraries, their translation units compiled in parallel."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, verbose, c) for c in (False, True)]
        return [f.result() for f in futs]


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib_path = LIB_CHECKED if checked else LIB
    out_dir = OUT_DIR_CHECKED if checked else OUT_DIR
    if not force and up_to_date(checked):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    exe = nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    defs = ["-DPKMOM_CHECKED=1"] if checked else []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [exe, *ARCH, *FLAGS, *defs, *inc, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources()), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib_path + f".{os.getpid()}.{int(checked)}.tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(exe)), "lib64")
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcufft", "-lcudart", "-Xlinker", f"-rpath={cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv, verbose=True))
