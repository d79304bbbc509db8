"""Measure the arithmetic peaks that bound this library's kernels on the
current GPU: FP64 DFMA (the roofline of the FP64 kernels), FP64 DMMA
(mma.sync), FP32 FFMA, and cuBLAS DGEMM / ZGEMM / TF32 SGEMM / CGEMM and an
HBM copy through torch, each timed with CUDA events after warm-up.

    python -m paper_1907_08560_gb300.peaks
"""
from __future__ import annotations

import ctypes


def probe(which: int, device: int = 0) -> float | None:
    from . import build
    lib = ctypes.CDLL(build.build_peak())
    lib.hzpeak_tflops.restype = ctypes.c_int
    lib.hzpeak_tflops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    t = ctypes.c_double(0.0)
    return t.value if lib.hzpeak_tflops(device, which, ctypes.byref(t)) == 0 else None


def _best(fn, reps=10):
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def library_peaks():
    import torch
    d = torch.device("cuda")
    out = {}
    n = 8192
    a = torch.randn(n, n, device=d, dtype=torch.float64)
    b = torch.randn(n, n, device=d, dtype=torch.float64)
    out["cublas_dgemm_tflops"] = 2 * n ** 3 / _best(lambda: a @ b, 3) / 1e9
    del a, b
    n = 4096
    a = torch.randn(n, n, device=d, dtype=torch.complex128)
    b = torch.randn(n, n, device=d, dtype=torch.complex128)
    out["cublas_zgemm_tflops"] = 8 * n ** 3 / _best(lambda: a @ b, 3) / 1e9
    del a, b
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    n = 8192
    a = torch.randn(n, n, device=d, dtype=torch.float32)
    b = torch.randn(n, n, device=d, dtype=torch.float32)
    out["cublas_sgemm_tf32_tflops"] = 2 * n ** 3 / _best(lambda: a @ b) / 1e9
    n = 4096
    a = torch.randn(n, n, device=d, dtype=torch.complex64)
    b = torch.randn(n, n, device=d, dtype=torch.complex64)
    out["cublas_cgemm_tf32_tflops"] = 8 * n ** 3 / _best(lambda: a @ b) / 1e9
    torch.backends.cuda.matmul.allow_tf32 = prev
    x = torch.empty(2 ** 30, dtype=torch.bfloat16, device=d)
    y = torch.empty_like(x)
    out["hbm_copy_gbs"] = 2 * 2 ** 31 / _best(lambda: y.copy_(x)) / 1e6
    return out


def main():
    res = {"fp64_dfma_tflops": probe(0), "fp64_dmma_tflops": probe(1), "fp32_ffma_tflops": probe(2)}
    res.update(library_peaks())
    for k, v in res.items():
        print(f"{k:28s} {v:10.3f}" if v is not None else f"{k:28s} failed")


if __name__ == "__main__":
    main()
