"""Drive the resident whole-run kernel (small embeddings) for timing and ncu.

    python -m paper_2303_05455_gb300.profile_resident --steps 1000 --reps 3
    ncu --set full --clock-control none -k regex:k_resident -s 1 -c 1 -o res \\
        python -m paper_2303_05455_gb300.profile_resident --steps 1000 --reps 2

Runs the gmm2k workload (2,000 vertices, exact kNN graph k = 2, r = 1) with
the resident kernel and with one launch per step, and prints the CUDA-event
time per step of each.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import ivhd, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--opt", default="momentum", choices=["momentum", "nesterov", "adadelta"])
    args = ap.parse_args()
    w = synth.WORKLOADS["gmm2k"]
    X, _ = synth.workload_features(w)
    knn = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k)
    s = torch.cuda.current_stream()
    for rep in range(args.reps):
        out = {"rep": rep}
        for resident in (True, "cluster", False):
            emb = ivhd.Embedding(knn, r=w.r, c=w.c, a=w.a, b=w.b, seed=w.seed, opt=args.opt,
                                 resident=resident)
            emb.step(16)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            emb.step(args.steps)
            e1.record(s)
            torch.cuda.synchronize()
            key = {True: "resident_us", "cluster": "cluster_us", False: "multi_launch_us"}[resident]
            out[key] = 1e3 * e0.elapsed_time(e1) / args.steps
            emb.close()
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
