"""Batched embeddings vs one-by-one FP32: 64 independent embeddings in one context.

    python -m paper_2303_05455_gb300.bench_batch [--n-emb 64] [--steps 1000]

Workload (synth.batch_workload): M log-uniform in [5,000, 200,000], N = 64
Gaussian mixtures with 5-30 components, k in {2, 3, 5, 10}, r in {1, 2},
c = 0.01, a = 0.9, b = 0.001, 1,000 momentum steps each.  The kNN graphs are
built on the GPU before anything is timed.  Timed, with CUDA events:

* one-by-one: for each embedding ivhd_create + 1,000 steps + positions, FP32;
* batched: one ivhd_create_batch with the launch shape (block size, hub
  threshold, vertices per warp) the autotuner chose beforehand + 1,000 steps (one launch per step
  for all embeddings) + positions, for BF16, FP16 and FP32 gathered
  positions; the library's default shape is reported beside it.

Prints one JSON line with both throughputs (edge-updates/s), the speed-up and
the kNN precision Q_NX(k) of every embedding under both runs.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import ivhd, synth


def measure(n_emb: int = 64, steps: int = 1000, qnx_rows: int = 2000,
            formats: str = "bf16,f16,f32") -> dict:
    """Runs the comparison and returns its figures as a dict (see the module docstring)."""
    args = argparse.Namespace(n_emb=n_emb, steps=steps, qnx_rows=qnx_rows, formats=formats)
    c, a, b = 0.01, 0.9, 0.001
    work = synth.batch_workload(n_emb=args.n_emb)
    t0 = time.perf_counter()
    graphs = [ivhd.knn_build(torch.from_numpy(w["X"]).cuda(), w["k"]) for w in work]
    torch.cuda.synchronize()
    knn_s = time.perf_counter() - t0
    s = torch.cuda.current_stream()

    def timed(fn):
        """fn(span) runs its embeddings, calling span() before each create and
        span() again once its positions are read back; the seconds of those
        spans are summed (create + steps + read-back; the contexts' teardown
        between them is not timed)."""
        evs = []

        def span():
            e = torch.cuda.Event(enable_timing=True)
            e.record(s)
            evs.append(e)

        torch.cuda.synchronize()
        out = fn(span)
        torch.cuda.synchronize()
        return out, sum(evs[q].elapsed_time(evs[q + 1]) for q in range(0, len(evs), 2)) / 1e3

    # one by one, FP32
    def one_by_one(span=lambda: None):
        pos, terms = [], 0
        for w, g in zip(work, graphs):
            span()
            emb = ivhd.Embedding(g, r=w["r"], c=c, a=a, b=b, seed=w["seed"])
            emb.step(args.steps)
            pos.append(emb.positions())
            span()
            terms += emb.info()["n_terms"]
            emb.close()
        return pos, terms

    one_by_one()  # warm-up (module load, graph instantiation paths)
    (pos1, terms), t_one = timed(one_by_one)

    # batched, autotuned, per gathered-position format
    lo = np.concatenate([[0], np.cumsum([w["X"].shape[0] for w in work])])
    sampled = [torch.from_numpy(synth.sample_rows(w["X"].shape[0], args.qnx_rows, e)).cuda()
               for e, w in enumerate(work)]
    q_one = [ivhd.eval_qnx(pos1[e], g, sampled[e]) for e, g in enumerate(graphs)]
    batched_runs = {}
    for fmt in args.formats.split(","):
        def create(shape=None):
            shape = shape or {"block": 0, "hub_threshold": 0, "vertices_per_warp": 0}
            return ivhd.Embedding.batch([g for g in graphs], r=[w["r"] for w in work],
                                        seeds=[w["seed"] for w in work], c=c, a=a, b=b,
                                        pos_format=fmt, block_size=shape["block"],
                                        hub_threshold=shape["hub_threshold"],
                                        vertices_per_warp=shape["vertices_per_warp"])

        emb0 = create()
        t = time.perf_counter()
        tuned = emb0.autotune(trial_steps=20)
        tune_s = time.perf_counter() - t
        emb0.close()

        def batched(span=lambda: None):
            span()
            emb = create(tuned)
            emb.step(args.steps)
            y = emb.positions()
            span()
            n = emb.info()["n_terms"]
            emb.close()
            return y, n

        def batched_untuned(span=lambda: None):
            span()
            emb = create()
            emb.step(args.steps)
            y = emb.positions()
            span()
            emb.close()
            return y

        batched()
        (ybat, terms_b), t_bat = timed(batched)
        _, t_plain = timed(batched_untuned)
        assert terms_b == terms
        dqs = [ivhd.eval_qnx(ybat[lo[e]:lo[e + 1]].contiguous(), g, sampled[e]) - q_one[e]
               for e, g in enumerate(graphs)]
        batched_runs[fmt] = {
            "seconds_tuned_shape": t_bat, "edge_updates_per_s": terms * args.steps / t_bat,
            "seconds_default_shape": t_plain, "autotune": tuned, "autotune_seconds": tune_s,
            "speedup_vs_one_by_one_f32": t_one / t_bat,
            "qnx_delta_vs_one_by_one": {"max_abs": max(abs(d) for d in dqs),
                                        "mean": float(np.mean(dqs))},
            "equal_precision": max(abs(d) for d in dqs) <= 0.01}

    line = {
        "workload": "64 embeddings, M log-uniform [5e3, 2e5], N=64 GMM 5-30 comps, k {2,3,5,10}, r {1,2}",
        "n_emb": args.n_emb, "total_M": int(lo[-1]), "steps": args.steps, "terms": terms,
        "one_by_one_f32": {"seconds": t_one, "edge_updates_per_s": terms * args.steps / t_one},
        "mean_qnx_one_by_one": float(np.mean(q_one)),
        "batched": batched_runs,
        "knn_build_s_untimed": knn_s,
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-emb", type=int, default=64)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--qnx-rows", type=int, default=2000)
    ap.add_argument("--formats", default="bf16,f16,f32")
    args = ap.parse_args()
    print(json.dumps(measure(args.n_emb, args.steps, args.qnx_rows, args.formats)), flush=True)


if __name__ == "__main__":
    main()
