"""Time the FP64-accurate tensor-core product on its own (one shape, CUDA events).

    python -m paper_2404_09373_gb300.gemm_bench --M 131072 --N 64 --K 832 --slices 8

The call goes through the C ABI (isdf_gemm_f64: slicing of both operands,
then the tcgen05 product), so the time includes the slicing kernels; a
profiler run with ``-k regex:k_oz_gemm`` isolates the product.  Inputs are
seeded normal numbers with a spread of row scales (like basis values and
factor rows); A is larger than the L2 cache at the default sizes.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=131072)
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--K", type=int, default=832)
    ap.add_argument("--slices", type=int, default=8)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    import torch

    from . import isdf as B

    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(1)
    A = torch.randn((a.M, a.K), generator=g, device=dev, dtype=torch.float64)
    A *= torch.exp2(torch.randint(-8, 8, (a.M, 1), generator=g, device=dev).to(torch.float64))
    Bm = torch.randn((a.N, a.K), generator=g, device=dev, dtype=torch.float64)
    C = torch.empty((a.M, a.N), device=dev, dtype=torch.float64)
    s = torch.cuda.current_stream()
    B.isdf_gemm_f64(A, Bm, C, slices=a.slices, stream=s.cuda_stream)  # warm-up
    ts = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        B.isdf_gemm_f64(A, Bm, C, slices=a.slices, stream=s.cuda_stream)
        e1.record(s)
        s.synchronize()
        ts.append(e0.elapsed_time(e1))
    ref = (A[:256].cpu().numpy() @ Bm.cpu().numpy().T)
    err = float(np.max(np.abs(C[:256].cpu().numpy() - ref)) / np.max(np.abs(ref)))
    ms = float(np.median(ts))
    print(json.dumps({"M": a.M, "N": a.N, "K": a.K, "slices": a.slices, "ms_call": ms,
                      "fp64_operand_gbs": 8.0 * a.M * a.K / ms / 1e6,
                      "fp64eq_tflops": 2.0 * a.M * a.N * a.K / ms / 1e9, "max_rel_err_vs_numpy": err}))


if __name__ == "__main__":
    main()
