"""Build the sm_103a shared library libghsvd.so in-tree with nvcc.

Each .cu translation unit is compiled in parallel, then linked with
``nvcc -shared``.  The library has a plain C ABI (include/ghsvd.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libghsvd.so")
PEAK_LIB = os.path.join(HERE, "libhzpeak.so")
SOURCES = ["ghsvd_api.cu", "hz_step.cu", "ghsvd_noalloc.cu", "hz_batch.cu", "hz_warm.cu",
           "hz_urv.cu", "hz_phase4.cu", "hz_tc.cu", "hz_delta.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "ghsvd.h"))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libghsvd.so."""
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_peak(force: bool = False) -> str:
    """Compile the FP64 peak probe (libhzpeak.so) used by the benchmark."""
    src = os.path.join(CSRC, "peak_probe.cu")
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= os.path.getmtime(src):
        return PEAK_LIB
    tmp = PEAK_LIB + ".tmp"
    r = subprocess.run([_nvcc(), *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", src, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for peak_probe.cu:\n{r.stderr}")
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build_peak(force=True))
