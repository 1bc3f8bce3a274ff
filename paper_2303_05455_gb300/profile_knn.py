"""Drive the kNN build for timing and ncu captures.

    python -m paper_2303_05455_gb300.profile_knn --data gmm --M 200000 --N 100 --reps 3
    python -m paper_2303_05455_gb300.profile_knn --data mnist --M 70000 --reps 3
    ncu --set full --clock-control none -k regex:k_knn_tc -s 1 -c 1 -o knn \\
        python -m paper_2303_05455_gb300.profile_knn --data mnist --M 70000 --reps 2

--data gmm: float32 Gaussian mixture (50 components, centres ~ N(0, 25 I));
--data mnist: uint8 MNIST-shaped images (784 pixels).  Prints, per repetition,
the wall time of ivhd_knn_build_ex (which synchronises) and the distance-GEMM
rate 2 M^2 K / t with K the padded operand width (3N for float, N for uint8).
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import ivhd, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", choices=["gmm", "mnist"], default="gmm")
    ap.add_argument("--M", type=int, default=200000)
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--method", default="tensor_cores", choices=sorted(ivhd.KNN_METHODS))
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    if args.data == "gmm":
        X, _ = synth.gaussian_mixture(args.M, args.N, 50, 11)
        K = -(-3 * args.N // 64) * 64
    else:
        X, _ = synth.mnist_like(args.M, 7, N=784)
        K = -(-784 // 64) * 64
    Xd = torch.from_numpy(X).cuda()
    for rep in range(args.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = ivhd.knn_build(Xd, args.k, method=args.method, return_stats=True)
        dt = time.perf_counter() - t0
        print(json.dumps({"rep": rep, "seconds": dt, "tflops": 2.0 * args.M ** 2 * K / dt / 1e12,
                          **st}), flush=True)


if __name__ == "__main__":
    main()
