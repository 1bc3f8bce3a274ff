"""Drive the warm-start network's training step and forward pass for timing and ncu.

    python -m paper_2303_05455_gb300.profile_mlp --steps 50
    ncu --metrics gpu__time_duration.sum --clock-control none --csv --log-file mlp.csv \\
        python -m paper_2303_05455_gb300.profile_mlp --steps 3

The MLP 784 -> 512 -> 512 -> 2 (GELU) takes Adam steps (lr 1e-3) on batches
of 4,096 random uint8 rows with random targets (shapes are what matter here),
then places 16,384 rows.  Prints CUDA-event milliseconds per training step,
the host enqueue time per step and the forward time.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import ivhd


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--batch", type=int, default=4096)
    args = ap.parse_args()
    B = args.batch
    net = ivhd.MLP(784, 512, max_batch=B)
    net.init_params(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randint(0, 256, (B * 4, 784), dtype=torch.uint8, device="cuda", generator=g)
    T = torch.randn((B * 4, 2), device="cuda", generator=g)
    for _ in range(3):
        net.train_step(X[:B], T[:B], lr=1e-3, x_scale=1 / 255)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = time.perf_counter()
    e0.record(s)
    for i in range(args.steps):
        b = (i % 4) * B
        net.train_step(X[b:b + B], T[b:b + B], lr=1e-3, x_scale=1 / 255)
    e1.record(s)
    host = time.perf_counter() - t
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(s)
    net.forward(X, x_scale=1 / 255)
    f1.record(s)
    torch.cuda.synchronize()
    print(json.dumps({"steps": args.steps, "gpu_ms_per_step": e0.elapsed_time(e1) / args.steps,
                      "host_ms_per_step_enqueue": 1e3 * host / args.steps,
                      "forward_rows": 4 * B, "forward_ms": f0.elapsed_time(f1)}), flush=True)
    net.close()


if __name__ == "__main__":
    main()
