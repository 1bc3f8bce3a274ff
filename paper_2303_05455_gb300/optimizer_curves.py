"""Stress against step for each optimiser and variant (the convergence comparison of
Sec. 3.3.2), on a GPU embedding, with the FP64 oracle's curve for momentum.

    python -m paper_2303_05455_gb300.optimizer_curves [--workload gmm2k] [--every 50]

Prints one JSON line: for momentum, Nesterov, Adadelta, momentum with
self-adaptive b, and momentum with an L1 final stage (last 50 steps), the
stress every `every` steps and the final Q_NX(k) and cf_10.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import ivhd, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gmm2k")
    ap.add_argument("--every", type=int, default=50)
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    X, labels = synth.workload_features(w)
    knn = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k)
    rows = torch.from_numpy(synth.sample_rows(w.M, 5000, 3)).cuda()
    runs = {
        "momentum": dict(opt="momentum"),
        "nesterov": dict(opt="nesterov"),
        "adadelta": dict(opt="adadelta"),
        "momentum_adaptive_b": dict(opt="momentum", adaptive=True),
        "momentum_l1_last50": dict(opt="momentum"),
    }
    out = {"workload": w.name, "n_iter": w.n_iter, "every": args.every, "curves": {}}
    for name, kw in runs.items():
        emb = ivhd.Embedding(knn, r=w.r, c=w.c, a=w.a, b=w.b, seed=w.seed, **kw)
        info = emb.info()
        curve = [emb.stress()]
        done = 0
        while done < w.n_iter:
            n = min(args.every, w.n_iter - done)
            if name == "momentum_l1_last50" and done + n > w.n_iter - 50 >= done:
                emb.step(w.n_iter - 50 - done)
                emb.set_metric("l1")
                emb.step(done + n - (w.n_iter - 50))
            else:
                emb.step(n)
            done += n
            if name == "momentum_l1_last50" and done > w.n_iter - 50:
                emb.set_metric("l2")
                curve.append(emb.stress())
                emb.set_metric("l1")
            else:
                curve.append(emb.stress())
        emb.set_metric("l2")
        y = emb.positions()
        rec = {"stress": curve, "qnx": ivhd.eval_qnx(y, knn, rows),
               "cf10": ivhd.eval_cf(y, labels, 10, rows), "max_degree": info["max_degree"]}
        if kw.get("adaptive"):
            rec["adaptive"] = emb.adaptive_state()
        out["curves"][name] = rec
        emb.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
