"""Build the CUDA library libfcofdm.so in-tree for sm_103a (nvcc, no cmake).

Usage: ``python -m paper_2008_00672_gb300.build`` or ``build()`` from Python.
The translation units are compiled in parallel and linked into
``paper_2008_00672_gb300/_build/libfcofdm.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfcofdm.so")
SOURCES = ["fc_kernels.cu", "fc_kernels_256.cu", "fc_kernels_128.cu", "fc_warp.cu", "fc_warp_cont.cu", "fc_plan.cu", "fc_static.cu", "fc_stream.cu", "fc_exec.cu",
           "fc_server.cu", "fc_tensor.cu", "fc_host.cu"]
# sources that include another source (fc_kernels.cu compiled for 256- and 128-thread CTAs)
INCLUDES = {"fc_kernels_256.cu": ["fc_kernels.cu"], "fc_kernels_128.cu": ["fc_kernels.cu"]}
HEADERS = ["fc_internal.cuh", "fc_device.cuh", "fc_tc.cuh", "fc_trace.h", "fc_warp_fft.cuh", os.path.join("..", "..", "include", "fcofdm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the FC library needs the CUDA toolkit to build")
    return cand


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS]
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    objs = [os.path.join(OUT_DIR, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    jobs = [(s, o) for s, o in zip(srcs, objs)
            if force or _stale(o, [s] + hdrs + [os.path.join(CSRC, d) for d in INCLUDES.get(os.path.basename(s), [])])]

    def compile_one(so):
        src, obj = so
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for msg in ex.map(compile_one, jobs):
            if verbose and msg:
                print(msg)
    if force or jobs or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcudart", "-ldl"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
