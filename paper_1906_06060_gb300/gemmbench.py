"""Micro-benchmark of the tcgen05 squeeze GEMM alone, through the C ABI (hotrg_gemm_split).

    python -m paper_1906_06060_gb300.gemmbench --M 10000 --N 40000 --K 10000 --npass 3 --reps 3

The default shape is one Dcut=10 chunk of the 4D squeeze with a quarter of its N range
(M = P = 10^4, N = 4 x 10^4, K = 10^4; about 3.6 GB of operands and output, so the working set
exceeds L2). Prints one JSON line: algorithmic TFLOP/s (2MNK per launch) and tensor-pipe
TFLOP/s (x npass), timed with CUDA events around the GEMM launches only (the FP32 -> bf16
plane split runs once, before timing).
"""
from __future__ import annotations

import argparse
import json
from ctypes import c_void_p

from . import _lib
from ._lib import check


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=10000)
    ap.add_argument("--N", type=int, default=40000)
    ap.add_argument("--K", type=int, default=10000)
    ap.add_argument("--npass", type=int, default=3)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--kblock", type=int, default=64)
    ap.add_argument("--fold-group", type=int, default=0)
    a = ap.parse_args()
    import torch
    lib = _lib.load()
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(0)
    A = torch.randn((a.M, a.K), device=dev, generator=g, dtype=torch.float32)
    Bt = torch.randn((a.N, a.K), device=dev, generator=g, dtype=torch.float32)
    C = torch.empty((a.M, a.N), device=dev, dtype=torch.float32)
    nbytes = lib.hotrg_gemm_scratch_bytes(a.M, a.N, a.K)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    args = lambda: (c_void_p(A.data_ptr()), A.stride(0), c_void_p(Bt.data_ptr()), Bt.stride(0),
                    c_void_p(C.data_ptr()), C.stride(0), a.M, a.N, a.K, a.npass, a.kblock, a.fold_group,
                    c_void_p(scratch.data_ptr()), nbytes, c_void_p(s.cuda_stream))
    check(lib.hotrg_gemm_split(*args()), "hotrg_gemm_split")   # warm-up (also splits planes)
    check(lib.hotrg_gemm_status(c_void_p(scratch.data_ptr()), c_void_p(s.cuda_stream)), "status")
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        check(lib.hotrg_gemm_split(*args()), "hotrg_gemm_split")
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    check(lib.hotrg_gemm_status(c_void_p(scratch.data_ptr()), c_void_p(s.cuda_stream)), "status")
    flops = 2.0 * a.M * a.N * a.K
    best = min(times)
    print(json.dumps({"M": a.M, "N": a.N, "K": a.K, "npass": a.npass, "kblock": a.kblock, "fold_group": a.fold_group, "ms": times,
                      "note": "timed region includes the plane split of A and Bt",
                      "alg_tflops": flops / (best * 1e-3) / 1e12,
                      "tensor_tflops": a.npass * flops / (best * 1e-3) / 1e12}))


if __name__ == "__main__":
    main()
