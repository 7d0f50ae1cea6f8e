"""Builds librve.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel and linked into
``paper_1610_03484_gb300/librve.so``; nothing is installed elsewhere.
``build(check=True)`` makes the checking build ``librve_check.so``
(-DRVE_BOUNDS_CHECK=1: DOF indices and columns tested before every gather and
scatter of the operator, residual and diagonal kernels) in its own folder.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librve.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "librve_check.so")
SOURCES = ["kernels.cu", "operator_tc.cu", "api.cu", "noalloc.cu", "surrogate.cu", "surrogate_api.cu", "macro.cu", "basis.cpp",
           "mesh.cpp", "partition.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librve")


def _compile(src: str, verbose: bool, build_dir: str = BUILD, defines=()) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3", *defines,
           "-I" + CSRC, "-I" + build_dir, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["-x", "cu"]
        if verbose:
            cmd.append("-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def gen_tables(build_dir: str = BUILD) -> None:
    """Compile and run the host generator of the compile-time basis tables."""
    os.makedirs(build_dir, exist_ok=True)
    exe = os.path.join(build_dir, "gen_tables")
    cxx = os.environ.get("CXX") or shutil.which("g++") or "c++"
    cmd = [cxx, "-O2", "-std=c++17", "-I" + CSRC, os.path.join(CSRC, "gen_tables.cpp"),
           os.path.join(CSRC, "basis.cpp"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"building gen_tables failed:\n{res.stderr}")
    res = subprocess.run([exe, os.path.join(build_dir, "basis_tables.inc")], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("gen_tables failed")


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile the library if any source is newer than it; returns its path.
    check=True builds the checking library librve_check.so instead."""
    lib, build_dir = (LIB_CHECK, BUILD_CHECK) if check else (LIB, BUILD)
    defines = ("-DRVE_BOUNDS_CHECK=1",) if check else ()
    srcs = [os.path.join(CSRC, s) for s in SOURCES + ["gen_tables.cpp"]]
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(os.path.dirname(HERE), "include", "rve.h"))
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(f) <= t for f in srcs + hdrs):
            return lib
    os.makedirs(build_dir, exist_ok=True)
    gen_tables(build_dir)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, build_dir, defines), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check="--check" in sys.argv))
