"""Learned warm start and out-of-sample placement, measured on the GPU.

    python -m paper_2303_05455_gb300.bench_warmstart [--holdout 1400000] [--epochs 10]

1. Train set: 200,000 MNIST-shaped points (synth.mnist_like, 784 uint8
   pixels); exact kNN graph (k = 5) and a plain IVHD embedding (r = 1,
   c = 0.01, momentum a = 0.9, b = 0.001, 2,000 steps).
2. The MLP 784 -> 512 -> 512 -> 2 (GELU) learns the standardised embedding
   with Adam (lr 1e-3, batch 4,096) on the library's tensor-core kernels.
3. Held-out set (default 1.4e6 points of the same distribution): the MLP
   places every point; IVHD then refines from that placement.  Compared with
   plain IVHD from a random start on the same graph, and with IVHD refining
   the nearest-neighbour placement (each point at the embedding of its
   nearest training point, the Progressive UMAP initialisation, Sec. 2.4.3;
   exact kNN query on the tensor cores): Q_NX(k), cf_10 and stress at
   checkpoints, and the steps each needs to come within 0.01 of plain IVHD's
   final kNN precision.
4. Arriving batches of 10,000 new points are placed by the MLP alone and by
   the nearest-neighbour placement: latency per batch and cf_10 of each new
   point against the training embedding (the share of its 10 nearest
   embedded training points with its own label).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import ivhd, synth


def measure(train: int = 200000, holdout: int = 1400000, epochs: int = 10, steps: int = 2000,
            check_every: int = 100, rows: int = 10000) -> dict:
    """Runs the comparison and returns its figures as a dict (see the module docstring)."""
    args = argparse.Namespace(train=train, holdout=holdout, epochs=epochs, steps=steps,
                              check_every=check_every, rows=rows)
    k, r, c, a, b = 5, 1, 0.01, 0.9, 0.001
    dev = torch.device("cuda")
    s = torch.cuda.current_stream()
    out = {"train": args.train, "holdout": args.holdout, "k": k, "r": r, "c": c, "b": b}

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(s)
        return e

    # 1. training embedding
    Xtr, Ltr = synth.mnist_like(args.train, 7, noise_seed=1)
    Xtr_d = torch.from_numpy(Xtr).to(dev)
    knn_tr = ivhd.knn_build(Xtr_d, k)
    emb = ivhd.Embedding(knn_tr, r=r, c=c, a=a, b=b, seed=11)
    emb.step(args.steps)
    Ytr = emb.positions()
    emb.close()
    mu, sd = Ytr.mean(0), Ytr.std(0)
    T = ((Ytr - mu) / sd).contiguous()

    # 2. MLP training (batches of 4,096); forward passes run in chunks of up to
    # max_batch rows, and chunks of 65,536 make the placement's GEMMs several
    # waves long (the outputs do not depend on the chunking)
    net = ivhd.MLP(784, 512, max_batch=65536)
    rng = np.random.Generator(np.random.PCG64(5))
    init = []
    for fo, fi, sc in ((512, 784, 1.0), (512, None, 0.0), (512, 512, 1.0), (512, None, 0.0),
                       (2, 512, 0.1), (2, None, 0.0)):
        if fi is None:
            init.append(np.zeros(fo))
        else:
            lim = np.sqrt(6.0 / fi)
            init.append(rng.uniform(-lim, lim, size=(fo, fi)).ravel() * sc)
    net.set_params(np.concatenate(init).astype(np.float32))
    B = 4096
    n_batches = args.train // B
    losses = []
    e0 = ev()
    for ep in range(args.epochs):
        perm = torch.from_numpy(rng.permutation(args.train)).to(dev)
        Xs, Ts = Xtr_d[perm].contiguous(), T[perm].contiguous()
        for bi in range(n_batches):
            sl = slice(bi * B, (bi + 1) * B)
            last = bi == n_batches - 1
            l = net.train_step(Xs[sl], Ts[sl], lr=1e-3, x_scale=1 / 255, want_loss=last)
            if last:
                losses.append(l)
    e1 = ev()
    torch.cuda.synchronize()
    train_s = e0.elapsed_time(e1) / 1e3
    out["mlp_train"] = {"epochs": args.epochs, "steps": args.epochs * n_batches,
                        "seconds": train_s,
                        "ms_per_step_with_shuffling": 1e3 * train_s / (args.epochs * n_batches),
                        "loss_last_batch_per_epoch": losses}

    # 3. held-out set: MLP placement, then IVHD refinement vs plain IVHD
    Xh, Lh = synth.mnist_like(args.holdout, 7, noise_seed=2)
    Xh_d = torch.from_numpy(Xh).to(dev)
    e0 = ev()
    Yp = net.forward(Xh_d, x_scale=1 / 255)
    e1 = ev()
    torch.cuda.synchronize()
    place_s = e0.elapsed_time(e1) / 1e3
    Yp = (Yp * sd + mu).contiguous()
    t = time.perf_counter()
    knn_h = ivhd.knn_build(Xh_d, k)
    torch.cuda.synchronize()
    out["holdout_knn_seconds_untimed"] = time.perf_counter() - t
    # the training set held as a kNN index (copied and prepared once)
    t = time.perf_counter()
    index = ivhd.KnnIndex(Xtr_d)
    torch.cuda.synchronize()
    index_s = time.perf_counter() - t
    e0 = ev()
    nn_h = index.query(Xh_d, 1)
    Ynn = ivhd.place_nn(Ytr, nn_h)
    e1 = ev()
    torch.cuda.synchronize()
    place_nn_s = e0.elapsed_time(e1) / 1e3
    rows = torch.from_numpy(synth.sample_rows(args.holdout, args.rows, 9)).to(dev)
    lab = torch.from_numpy(Lh).to(dev)

    def run(init_pos):
        e = ivhd.Embedding(knn_h, r=r, c=c, a=a, b=b, seed=13, init_uniform=init_pos is None)
        if init_pos is not None:
            e.set_positions(init_pos)
        curve = []
        y = e.positions()
        curve.append({"step": 0, "qnx": ivhd.eval_qnx(y, knn_h, rows),
                      "cf10": ivhd.eval_cf(y, lab, 10, rows), "stress": e.stress()})
        secs = 0.0
        for st in range(args.check_every, args.steps + 1, args.check_every):
            t0 = ev()
            e.step(args.check_every)
            t1 = ev()
            torch.cuda.synchronize()
            secs += t0.elapsed_time(t1) / 1e3
            y = e.positions()
            curve.append({"step": st, "qnx": ivhd.eval_qnx(y, knn_h, rows),
                          "cf10": ivhd.eval_cf(y, lab, 10, rows), "stress": e.stress()})
        e.close()
        return curve, secs, y

    plain, plain_s, _ = run(None)
    warm, warm_s, _ = run(Yp)
    nnw, nnw_s, _ = run(Ynn)
    q_final = plain[-1]["qnx"]

    def first_within(curve):
        for pt in curve:
            if abs(pt["qnx"] - q_final) <= 0.01 and pt["qnx"] >= q_final - 0.01:
                return pt["step"]
        return None

    out["placement"] = {"rows": args.holdout, "seconds": place_s,
                        "rows_per_s": args.holdout / place_s, "mlp_launches": net.launches()}
    out["plain_ivhd"] = {"curve": plain, "step_seconds": plain_s,
                         "steps_to_final_precision": first_within(plain)}
    out["warm_start_ivhd"] = {"curve": warm, "step_seconds": warm_s,
                              "steps_to_plain_final_precision": first_within(warm)}
    out["nn_placement"] = {"rows": args.holdout, "seconds": place_nn_s,
                           "rows_per_s": args.holdout / place_nn_s,
                           "index_create_seconds": index_s,
                           "what": "exact 1-NN query in the training set (a KnnIndex built "
                                   "once) + its embedding"}
    out["nn_placement_ivhd"] = {"curve": nnw, "step_seconds": nnw_s,
                                "steps_to_plain_final_precision": first_within(nnw)}

    # 4. arriving batches, assessed against the training embedding they are placed into
    Xa, La = synth.mnist_like(10 * 10000, 7, noise_seed=3)
    Xa_d = torch.from_numpy(Xa).to(dev)
    La_d = torch.from_numpy(La).to(dev)
    Ltr_d = torch.from_numpy(Ltr).to(dev)

    def cf_vs_train(yb, lb):
        nb = ivhd.knn_query(yb.contiguous(), Ytr, 10).long()
        return float((Ltr_d[nb] == lb[:, None]).float().mean())

    res = {"mlp": {"latency_us": [], "cf10": []}, "nn": {"latency_us": [], "cf10": []}}
    for bi in range(10):
        xb = Xa_d[bi * 10000:(bi + 1) * 10000].contiguous()
        lb = La_d[bi * 10000:(bi + 1) * 10000]
        t0 = ev()
        yb = net.forward(xb, x_scale=1 / 255)
        t1 = ev()
        torch.cuda.synchronize()
        res["mlp"]["latency_us"].append(t0.elapsed_time(t1) * 1e3)
        res["mlp"]["cf10"].append(cf_vs_train(yb * sd + mu, lb))
        t0 = ev()
        yn = ivhd.place_nn(Ytr, index.query(xb, 1))
        t1 = ev()
        torch.cuda.synchronize()
        res["nn"]["latency_us"].append(t0.elapsed_time(t1) * 1e3)
        res["nn"]["cf10"].append(cf_vs_train(yn, lb))
    rows_tr = torch.from_numpy(synth.sample_rows(args.train, args.rows, 9)).to(dev)
    out["arriving_batches"] = {"batch": 10000, "placed_by": res,
                               "train_embedding_cf10": ivhd.eval_cf(Ytr, Ltr_d, 10, rows_tr)}
    # the Adam step alone (last, so the network used above is not changed):
    # 50 steps on resident batches, no shuffling in between
    Xs, Ts = Xtr_d[:4 * B].contiguous(), T[:4 * B].contiguous()
    torch.cuda.synchronize()
    e2 = ev()
    for i in range(50):
        net.train_step(Xs[(i % 4) * B:(i % 4 + 1) * B], Ts[(i % 4) * B:(i % 4 + 1) * B], lr=1e-3,
                       x_scale=1 / 255)
    e3 = ev()
    torch.cuda.synchronize()
    out["mlp_train"]["ms_per_step"] = e2.elapsed_time(e3) / 50
    refine = min(len(warm) - 1, max(1, 100 // args.check_every))
    out["summary"] = {
        "train_step_ms": out["mlp_train"]["ms_per_step"],
        "placement_s": place_s,
        "batch_10k_ms": {"mlp": float(np.median(res["mlp"]["latency_us"])) / 1e3,
                         "nn": float(np.median(res["nn"]["latency_us"])) / 1e3},
        "stress": {"plain_start": plain[0]["stress"], "warm_start": warm[0]["stress"],
                   f"warm_after_{warm[refine]['step']}_steps": warm[refine]["stress"],
                   f"plain_after_{plain[-1]['step']}_steps": plain[-1]["stress"],
                   f"warm_after_{warm[-1]['step']}_steps": warm[-1]["stress"]},
        "qnx_final": {"plain": plain[-1]["qnx"], "warm": warm[-1]["qnx"], "nn": nnw[-1]["qnx"]},
        "equal_precision": abs(warm[-1]["qnx"] - plain[-1]["qnx"]) <= 0.01,
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200000)
    ap.add_argument("--holdout", type=int, default=1400000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--rows", type=int, default=10000)
    args = ap.parse_args()
    print(json.dumps(measure(args.train, args.holdout, args.epochs, args.steps, args.check_every,
                             args.rows)), flush=True)


if __name__ == "__main__":
    main()
