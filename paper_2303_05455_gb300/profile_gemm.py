"""Drive the tcgen05 BF16 GEMM for timing and ncu captures.

    python -m paper_2303_05455_gb300.profile_gemm [--shapes 8192x8192x8192,4096x512x784]

Each shape M x N x K runs `--reps` times through ivhd_gemm_bf16_tn (C = A B^T,
FP32 out); prints the CUDA-event time per call (which includes the call's
small set-up and read-back of its error flag) and the resulting TFLOP/s.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import ivhd


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shapes", default="8192x8192x8192,4096x512x784,4096x512x512,512x784x4096")
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    s = torch.cuda.current_stream()
    res = []
    for sh in args.shapes.split(","):
        M, N, K = (int(v) for v in sh.split("x"))
        g = torch.Generator(device="cuda").manual_seed(M + N + K)
        A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
        ivhd.gemm_bf16_tn(A, B)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.reps):
            C = ivhd.gemm_bf16_tn(A, B)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        ref = (A[:64].float() @ B.float().T)
        err = float((C[:64] - ref).abs().max() / ref.abs().max())
        res.append({"M": M, "N": N, "K": K, "ms_per_call": ms,
                    "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12, "max_rel_err_rows0_63": err})
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
