"""Build the CUDA library in-tree: ``_build/liblacos.so`` for sm_103a.

The kernels must be compiled without FMA contraction and with IEEE division
and square root, so that results match the float32 definition bit for bit.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblacos.so")
PEAK_LIB = os.path.join(OUT_DIR, "libalupeak.so")
SOURCES = ["lacos.cu"]
DEPS = ["lacos_kernels.cuh", "networks.cuh", "gain_math.cuh", os.path.join("..", "..", "include", "lacos.h")]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false",
    "-Xcompiler", "-fPIC", "-shared",
    "-Xptxas", "-v",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(lib, files) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(os.path.join(CSRC, f)) > t for f in files)


def _compile(lib, sources, log_name, verbose):
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + NVCC_FLAGS + [os.path.join(CSRC, s) for s in sources] + ["-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"nvcc failed building {os.path.basename(lib)}")
    with open(os.path.join(OUT_DIR, log_name), "w") as f:
        f.write(res.stderr)
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liblacos.so and the benchmark's libalupeak.so (in parallel) if stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = []
    if force or _stale(LIB, SOURCES + DEPS):
        jobs.append((LIB, SOURCES, "ptxas.log"))
    if force or _stale(PEAK_LIB, ["alu_peak.cu"]):
        jobs.append((PEAK_LIB, ["alu_peak.cu"], "ptxas_alupeak.log"))
    if jobs:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(len(jobs)) as ex:
            for fut in [ex.submit(_compile, lib, src, log, verbose) for lib, src, log in jobs]:
                fut.result()
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
