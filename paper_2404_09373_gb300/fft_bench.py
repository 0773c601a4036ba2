"""Time the double-float 3-D transform on its own (one shape, CUDA events), next
to torch.fft.rfftn (cuFFT, FP64) on the same grids.

    python -m paper_2404_09373_gb300.fft_bench --nx 96 --ny 96 --nz 96 --batch 37

Prints per-vector times, the effective traffic (input + output once) and the
largest difference between the two results relative to the grid's l1 norm.
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=96)
    ap.add_argument("--ny", type=int, default=96)
    ap.add_argument("--nz", type=int, default=96)
    ap.add_argument("--batch", type=int, default=37)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    import torch

    from . import isdf as B

    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(1)
    f = torch.randn((a.batch, a.nz, a.ny, a.nx), generator=g, device=dev, dtype=torch.float64)
    S = torch.empty((a.batch, a.nz, a.ny, a.nx // 2 + 1), dtype=torch.complex128, device=dev)
    s = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(a.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            s.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    ms_df = timed(lambda: B.isdf_rfft3(f, S, stream=s.cuda_stream))
    ref = None

    def cufft():
        nonlocal ref
        ref = torch.fft.rfftn(f, dim=(1, 2, 3))

    ms_cu = timed(cufft)
    err = float(((S - ref).abs().amax(dim=(1, 2, 3)) / f.abs().sum(dim=(1, 2, 3))).max())
    nbytes = a.batch * (8 * a.nx * a.ny * a.nz + 16 * (a.nx // 2 + 1) * a.ny * a.nz)
    print(json.dumps({"shape": [a.nx, a.ny, a.nz], "batch": a.batch, "us_per_vector_double_float": 1e3 * ms_df / a.batch,
                      "us_per_vector_cufft_fp64": 1e3 * ms_cu / a.batch,
                      "effective_gbs_double_float": nbytes / ms_df / 1e6, "max_err_rel_l1": err}))


if __name__ == "__main__":
    main()
