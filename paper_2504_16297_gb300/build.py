"""Builds libptsbe.so in-tree: host C++ with g++, CUDA with nvcc for sm_103a only."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libptsbe.so")

CXX_SOURCES = ["api.cpp", "pts.cpp", "circuit.cpp", "backward.cpp", "dense_plan.cpp"]
CU_SOURCES = ["evolve.cu", "sample.cu", "pershot.cu", "backward.cu", "dense.cu"]
HEADERS = ["internal.h", "philox.h", "tile_ops.cuh", "frame.cuh", "dense.cuh", "fixed_point.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: the PTSBE library needs the CUDA toolkit to build")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in CXX_SOURCES + CU_SOURCES + HEADERS]
    paths.append(os.path.join(INCLUDE, "ptsbe.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every translation unit in parallel and links libptsbe.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", CSRC, "-I", INCLUDE, "-I", os.path.join(cuda, "include")]
    jobs = []
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append((["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-fvisibility=hidden",
                      "-Wall", "-Wno-unknown-pragmas", *inc, "-c", os.path.join(CSRC, f), "-o", obj], obj))
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append(([nvcc, *ARCH, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
                      "-Xcompiler", "-fvisibility=hidden", "-Xptxas", "-v" if verbose else "-O3", *inc,
                      "-c", os.path.join(CSRC, f), "-o", obj], obj))

    def run(job):
        cmd, _ = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    for cmd, r in results:
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *[o for _, o in jobs]]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
