"""Build the CUDA library in-tree with nvcc (sm_103a only).

Produces ``paper_1809_01334_gb300/_build/libocraycast.so`` from the sources in
``csrc/``, and ``_build/libocrpeak.so`` (the FP32 FMA throughput
microbenchmark that the benchmark's roofline is set against) from
``csrc/ocr_fp32_peak.cu``.  Translation units compile in parallel; each
library is linked by one nvcc call.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libocraycast.so")
SOURCES = ["ocr_capi.cu", "ocr_kernels.cu", "ocr_batch.cu", "ocr_backward.cu", "ocr_shell.cu"]
PEAK_SOURCE = "ocr_fp32_peak.cu"
PEAK_LIB = os.path.join(OUT_DIR, "libocrpeak.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: -ffp-contract=off keeps the FP64 tables (plane tangents, radii) as
# written, so that their rounding to float is the same on every host
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler",
         "-ffp-contract=off", "--use_fast_math", "-Xptxas", "-v"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "ocraycast.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    dep = _deps()
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= dep
            and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= dep):
        return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    peak_obj = None
    with cf.ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        for src, (obj, log) in zip(SOURCES + [PEAK_SOURCE],
                                   ex.map(compile_one, SOURCES + [PEAK_SOURCE])):
            if src == PEAK_SOURCE:
                peak_obj = obj
            else:
                objs.append(obj)
            if verbose:
                print(log)
    for out, ins in ((LIB, objs), (PEAK_LIB, [peak_obj])):
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *ins]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
