"""FP64 throughput of this GPU, the roof of the FP64-storage step (bound by the
FP64 pipe, not by HBM): a cuBLAS DGEMM through torch, n = 8192, best of the
timed repetitions after two warm-up products.

    python -m paper_2011_06856_gb300.peaks
"""
from __future__ import annotations

import json


def dgemm_tflops(n: int = 8192, reps: int = 5) -> float:
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


if __name__ == "__main__":
    print(json.dumps({"fp64_dgemm_tflops": dgemm_tflops()}))
