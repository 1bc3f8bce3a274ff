"""Drive the fused step kernel on a full-size workload, for timing and ncu captures.

    python -m paper_2303_05455_gb300.profile_step --graph knn --iters 200
    ncu --set full --clock-control none -k regex:k_step -s 10 -c 1 \\
        -o prof python -m paper_2303_05455_gb300.profile_step --graph knn --iters 20

``--graph knn`` builds the exact kNN graph of the gmm1p4m workload on the GPU
(about 20 s, once); ``--graph random`` uses a kNN-shaped random graph with
hubs of the same size.  Prints create time and CUDA-event time per step.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import ivhd, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gmm1p4m", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--graph", choices=["knn", "random"], default="knn")
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--opt", default="momentum", choices=["momentum", "nesterov", "adadelta"])
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    if args.graph == "knn":
        X, _ = synth.workload_features(w)
        Xd = torch.from_numpy(X).cuda()
        knn = ivhd.knn_build(Xd, w.k)
        del Xd
    else:
        knn = torch.from_numpy(synth.random_knn_graph(w.M, w.k, w.seed + 1, hub_frac=0.02,
                                                      n_hubs=max(w.k + 1, w.M // 1000))).cuda()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    for rep in range(args.reps):
        t0 = time.perf_counter()
        emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=args.opt, a=w.a, b=w.b, seed=w.seed)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        emb.step(args.iters)
        e1.record(s)
        torch.cuda.synchronize()
        info = emb.info()
        emb.close()
        print(json.dumps({"rep": rep, "create_ms": 1e3 * (t1 - t0),
                          "us_per_step": 1e3 * e0.elapsed_time(e1) / args.iters,
                          "n_hub": info["n_hub"], "nnz_sym": info["nnz_sym"],
                          "max_degree": info["max_degree"]}), flush=True)


if __name__ == "__main__":
    main()
