"""Measured tensor and FP64 peaks of the current GPU, the denominators of the
TF32-form and FP64-form rooflines.

* TF32 tensor: torch.matmul of float32 8192 x 8192 matrices with TF32 tensor
  cores allowed (cuBLAS), 2 N^3 flops: best of 10 (burst) and back to back for
  4 s (sustained).
* FP64: torch.matmul of float64 4096 x 4096 matrices (cuBLAS DGEMM), best of 5
  and back to back for 4 s; and the CUDA-core FMA rate of the repo's own probe
  (probes/dfma.cu: independent FMA chains on every SM), the bound of the FP64
  form's hand-written contraction.

  python -m paper_2203_05632_gb300.peaks [--seconds 4]   (prints one JSON line)
"""
from __future__ import annotations

import argparse
import ctypes
import json
import time


def _matmul_rate(torch, n, dtype, reps, seconds):
    a = torch.randn(n, n, device="cuda", dtype=dtype)
    b = torch.randn(n, n, device="cuda", dtype=dtype)
    c = torch.empty(n, n, device="cuda", dtype=dtype)
    torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    flops = 2.0 * n ** 3
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    # sustained: back to back for `seconds`
    k = max(1, int(seconds * best * 1e12 / flops))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(k):
        torch.matmul(a, b, out=c)
    e1.record()
    e1.synchronize()
    sustained = k * flops / (e0.elapsed_time(e1) / 1e3) / 1e12
    return best, sustained


def measure(seconds: float = 4.0, device: int = 0) -> dict:
    import torch

    from .build import build_probes
    torch.cuda.set_device(device)
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        tf32_burst, tf32_sust = _matmul_rate(torch, 8192, torch.float32, 10, seconds)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    f64_burst, f64_sust = _matmul_rate(torch, 4096, torch.float64, 5, seconds)
    lib = ctypes.CDLL(build_probes())
    lib.probe_dfma_tflops.restype = ctypes.c_int
    lib.probe_dfma_tflops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double)]
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    scratch = torch.empty(sms * 8 * 256, dtype=torch.float64, device="cuda")
    dfma = ctypes.c_double(0.0)
    rc = lib.probe_dfma_tflops(device, 8, 1.0, ctypes.c_void_p(scratch.data_ptr()), ctypes.byref(dfma))
    if rc != 0:
        raise RuntimeError(f"DFMA probe failed with CUDA error {rc}")
    return {"tf32_tflops": tf32_burst, "tf32_tflops_sustained": tf32_sust,
            "fp64_dgemm_tflops": f64_burst, "fp64_dgemm_tflops_sustained": f64_sust,
            "fp64_fma_tflops": dfma.value, "gpu": torch.cuda.get_device_name(device),
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
            "how": "torch.matmul fp32 8192^3 with TF32 allowed and fp64 4096^3 (best of 10 / 5, and back to "
                   "back for %g s); probes/dfma.cu: 8 independent FMA chains per thread, 8 x 256-thread "
                   "blocks per SM, best of 8 launches" % seconds}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--seconds", type=float, default=4.0)
    args = ap.parse_args()
    print(json.dumps(measure(args.seconds)))


if __name__ == "__main__":
    main()
