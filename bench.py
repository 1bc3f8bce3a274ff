#!/usr/bin/env python3
"""IVHD benchmark: edge-updates/s and seconds-to-embed on one GB300.

One timed step is one whole embedding of the workload (default ``gmm1p4m``:
M = 1.4e6 points, N = 100, k = 5, r = 1, c = 0.01, 2,000 momentum steps):
``ivhd_create`` (random neighbours, symmetric layout, initial positions) +
``ivhd_step(2000)`` + positions read-back, all through the C ABI with the kNN
graph already resident in HBM (the context's teardown follows the timed
region).  The exact kNN graph is built once before the
timed region (untimed, as the paper's time_emb excludes the graph build).

    value = terms x iterations / seconds per embedding      (edge-updates/s)

``e2e`` repeats the step from pinned host memory (kNN upload and positions
download inside the timed region).  ``roofline`` reports the fused step
kernel against the measured HBM copy bandwidth.  ``cpu_baseline`` times the
FP64 oracle on a bounded sample of the same workload on one core, and
``cpu_baseline.all_cores`` the same loop on every host core.

``--impl reference`` times the FP64 CPU oracle (the only reference this
project has) on the same metric; under torchrun only rank 0 runs it.

Besides the headline, the line carries the other workloads, each timed on
its own with its clocks (``--no-extras`` skips them):

* ``configs.gmm2k`` and ``configs.mnist70k`` (momentum and Adadelta): the same
  whole-embedding step, its kernel time per iteration against the measured
  random-gather bound, Q_NX / cf / stress of the result;
* ``batch64``: 64 embeddings of uneven size in one context (FP32 / FP16 /
  BF16 gathered positions, autotuned launch shape) against one-by-one FP32;
* ``warmstart``: the learned warm start (training step, placement of a
  1.4e6-point held-out set and of 10,000-point batches, IVHD refinement)
  against plain IVHD from the uniform start.

``--kernel step|knn|gemm|mlp|resident`` runs one kernel family alone (for
timing and ncu captures) and prints its CUDA-event timings as JSON lines.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2303_05455_gb300 import synth  # noqa: E402

METRIC = "IVHD edge-updates/s & s-to-embed @M=1.4M vs plain FP32, at equal kNN precision"
UNIT = "edge-updates/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="gmm1p4m", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--opt", default="momentum", choices=["momentum", "nesterov", "adadelta"],
                    help="optimiser of the step (Sec. 3.3.2 / 3.3.3)")
    ap.add_argument("--n-iter", type=int, default=None, help="iterations per embedding")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU seconds of the oracle baseline sample")
    ap.add_argument("--variants", default="f16,bf16,f32:degree_cluster,f16:degree_cluster,"
                                          "bf16:degree_cluster",
                    help="position formats / layout orders also timed, format[:order] "
                         "(comma list, or 'none')")
    ap.add_argument("--qnx-rows", type=int, default=10000)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the gmm2k / mnist70k / batch64 / warmstart sub-objects")
    cap = ap.add_argument_group("kernel capture modes (--kernel)")
    cap.add_argument("--kernel", choices=["step", "knn", "gemm", "mlp", "resident"], default=None)
    cap.add_argument("--graph", choices=["knn", "random"], default="knn",
                     help="step: the workload's exact kNN graph or a kNN-shaped random graph")
    cap.add_argument("--iters", type=int, default=200, help="step: iterations per repetition")
    cap.add_argument("--reps", type=int, default=2)
    cap.add_argument("--pos-format", default="f32",
                     help="step: gathered position formats, comma list of f32, f16, bf16")
    cap.add_argument("--order", default="degree",
                     help="step: layout orders, comma list of degree, degree_cluster")
    cap.add_argument("--shapes-step", default="0:0:0",
                     help="step: launch shapes hub_threshold:vertices_per_warp:block_size"
                          "[:form], comma list (0 = library default; form auto, multi, "
                          "grid, cluster, block)")
    cap.add_argument("--data", choices=["gmm", "mnist"], default="gmm", help="knn: data set")
    cap.add_argument("--M", type=int, default=200000, help="knn: rows")
    cap.add_argument("--N", type=int, default=100, help="knn: float dimensions")
    cap.add_argument("--shapes", default="8192x8192x8192,4096x512x784,4096x512x512,512x784x4096",
                     help="gemm: M x N x K list")
    cap.add_argument("--batch", type=int, default=4096, help="mlp: batch rows")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def workload_config(w: synth.Workload, n_iter: int, opt: str = "momentum") -> dict:
    return {
        "workload": w.name, "M": w.M, "N": w.N, "features": w.dtype, "k": w.k, "r": w.r,
        "c": w.c, "n_iter": n_iter, "optimizer": opt, "a": w.a, "b": w.b,
        "terms": "multiplicity (mutual kNN pairs give two nn terms)",
        "step": "ivhd_create + n_iter fused steps + positions read-back (one embedding)",
        "knn_graph": "exact, built on the GPU before the timed region (untimed)",
        "l2": "256 MiB buffer written between timed steps; the per-iteration working "
              "set (~110 MB) stays in L2 within an embedding",
    }


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region.

    The sampler starts, and its first sample is awaited, before the timed
    region opens, so that nvidia-smi's own start-up does not overlap the timed
    work; a reader thread drains its output while it runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, first_sample_timeout: float = 10.0):
        import threading

        self.proc = None
        self.gpu = gpu_index
        self.lines = []
        self._first = threading.Event()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._reader = threading.Thread(target=self._drain, daemon=True)
        self._reader.start()
        self._first.wait(first_sample_timeout)
        self.n_before = len(self.lines)   # samples taken before the timed region

    def _drain(self):
        for line in self.proc.stdout:
            self.lines.append(line)
            self._first.set()
        self._first.set()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self._reader.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the samples of the timed region (the last one before it opened included,
        # so that a short region still has one)
        for line in self.lines[max(0, self.n_before - 1):]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def step_kernel_traffic():
    """dram bytes per launch of the step kernel from the committed ncu summary,
    only while the kernel source is unchanged since the capture."""
    src = os.path.join(ROOT, "paper_2303_05455_gb300", "csrc", "ivhd_step.cu")
    meta = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        with open(meta) as f:
            d = json.load(f)
        if d.get("kernel_src_sha256") == sha and d.get("workload"):
            return d
    except (OSError, ValueError):
        pass
    return None


def aggregate_ranks(total_s: float, kernel_ms: float, units: float, device) -> tuple:
    """Whole-job figures over the ranks of the default process group: the max
    of the timed seconds and of the kernel time, the sum of the units."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([total_s, kernel_ms, units], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(t[2])


# ------------------------------------------------------------- oracle leg


ORACLE_OPT = {"momentum": 0, "nesterov": 1, "adadelta": 2}


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(w: synth.Workload, target_s: float, max_iters: int = 200, opt: str = "momentum",
                  threads: int = 1):
    """Times the FP64 oracle's step loop on a graph of the workload's shape.

    The graph comes from the input generators (a kNN-shaped graph with hubs,
    M x k), not from the GPU path.  The serial loop (oracle.run) is timed for
    about target_s seconds, then, with threads > 1, the same loop on that many
    host threads (oracle.run_threads) for about as long.  Returns a dict with
    edge-updates/s, iterations and seconds of each, the term count and the
    set-up seconds.
    """
    import oracle

    t0 = time.perf_counter()
    knn = synth.random_knn_graph(w.M, w.k, w.seed + 1, hub_frac=0.02, n_hubs=max(w.k + 1, w.M // 1000))
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    out = {"terms": terms.T, "setup_s": time.perf_counter() - t0}

    def timed(fn):
        t = time.perf_counter()
        fn(st, terms, w.c, 1)
        one = max(time.perf_counter() - t, 1e-6)
        iters = int(max(1, min(max_iters, target_s / one)))
        t = time.perf_counter()
        fn(st, terms, w.c, iters)
        dt = time.perf_counter() - t
        return {"value": terms.T * iters / dt, "iters": iters, "seconds": dt}

    out["serial"] = timed(lambda s_, t_, c_, n_: oracle.run(s_, t_, c_, n_, ORACLE_OPT[opt],
                                                            a=w.a, b=w.b))
    if threads > 1:
        out["threads"] = timed(lambda s_, t_, c_, n_: oracle.run_threads(
            s_, t_, c_, n_, ORACLE_OPT[opt], a=w.a, b=w.b, threads=threads))
        out["threads"]["cores"] = threads
    return out


def run_reference(args):
    if not hasattr(args, "opt"):
        args.opt = "momentum"
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    w = synth.WORKLOADS[args.workload]
    n_iter = args.n_iter or w.n_iter
    import oracle

    knn = synth.random_knn_graph(w.M, w.k, w.seed + 1, hub_frac=0.02, n_hubs=max(w.k + 1, w.M // 1000))
    rn, _ = oracle.random_neighbors(knn, w.r, w.seed)
    terms = oracle.build_terms(knn, rn)
    st = oracle.State.fresh(oracle.init_positions(w.M, w.seed))
    t = time.perf_counter()
    oracle.run(st, terms, w.c, 1, ORACLE_OPT[args.opt], a=w.a, b=w.b)
    one = max(time.perf_counter() - t, 1e-6)
    per_step = int(max(1, min(n_iter, 6.0 / one)))   # ~6 s of oracle work per step
    for _ in range(args.warmup):
        oracle.run(st, terms, w.c, per_step, ORACLE_OPT[args.opt], a=w.a, b=w.b)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.run(st, terms, w.c, per_step, ORACLE_OPT[args.opt], a=w.a, b=w.b)
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = terms.T * per_step / (ms / 1e3)
    sample = (f"{per_step} of {n_iter} iterations per step on a {w.M} x {w.k} kNN-shaped "
              f"graph from the input generators (r={w.r}), FP64, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {**workload_config(w, n_iter, args.opt),
                                         "iterations_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU leg


def run_ours(args):
    import torch

    from paper_2303_05455_gb300 import ivhd

    rank, local_rank, world = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for the GPU leg")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    w = synth.WORKLOADS[args.workload]
    n_iter = args.n_iter or w.n_iter

    # untimed set-up: data, exact kNN graph (replicas: every rank embeds its own copy)
    X, labels = synth.workload_features(w)
    Xd = torch.from_numpy(X).to(dev)
    t = time.perf_counter()
    knn = ivhd.knn_build(Xd, w.k)
    torch.cuda.synchronize()
    knn_seconds = time.perf_counter() - t
    del Xd, X
    torch.cuda.empty_cache()

    stream = torch.cuda.current_stream()
    out = torch.empty((w.M, 2), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def one_embedding(knn_in, out_buf, evs=None, pos_format="f32", order="degree",
                      after_readback=None):
        """create + n_iter steps + positions read-back; after_readback() marks the end
        of the timed embedding (the context's teardown follows it)."""
        emb = ivhd.Embedding(knn_in, r=w.r, c=w.c, opt=args.opt, a=w.a, b=w.b, seed=w.seed,
                             stream=stream, device=dev, pos_format=pos_format, order=order)
        if evs is not None:
            evs[0].record(stream)
        emb.step(n_iter)
        if evs is not None:
            evs[1].record(stream)
        emb.positions(out=out_buf)
        if after_readback is not None:
            after_readback()
        info = emb.info()
        emb.close()
        return info

    for _ in range(args.warmup):
        info = one_embedding(knn, out)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    launches = 0
    clocks = ClockSampler(local_rank) if rank == 0 else None
    gc.collect()
    gc.disable()   # no collector pauses between the host calls of a timed embedding
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        starts[s].record(stream)
        info = one_embedding(knn, out, kev[s], after_readback=lambda: ends[s].record(stream))
        launches += info["setup_launches"] + info["kernel_launches"] + info["aux_launches"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    gc.enable()
    clk = clocks.stop() if clocks else None
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    ms = statistics.mean(step_ms)
    kms = statistics.mean(kern_ms)
    terms = info["n_terms"]
    units = terms * n_iter * args.steps

    if world > 1:
        total_s, kms, total_units = aggregate_ranks(sum(step_ms) / 1e3, kms, float(units), dev)
    else:
        total_s, total_units = sum(step_ms) / 1e3, float(units)
    value = total_units / total_s

    # kNN precision of the timed embedding (sampled rows, exact neighbour sets),
    # class purity cf_nn, stress and finiteness of the final positions
    # Q_NX / cf over every vertex up to 1e5 vertices, else over a seeded sample
    if w.M <= 100_000:
        rows = torch.arange(w.M, dtype=torch.int64, device=dev)
    else:
        rows = torch.from_numpy(synth.sample_rows(w.M, args.qnx_rows, 12345)).to(dev)
    lab = torch.from_numpy(labels).to(dev)

    def quality(pos_format="f32", order="degree"):
        emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=args.opt, a=w.a, b=w.b, seed=w.seed,
                             stream=stream, device=dev, pos_format=pos_format, order=order)
        emb.step(n_iter)
        emb.positions(out=out)
        try:
            E, finite = emb.stress(), True
        except ivhd.IvhdError:
            E, finite = float("nan"), False
        emb.close()
        return {"qnx": ivhd.eval_qnx(out, knn, rows),
                "cf": {str(nn): ivhd.eval_cf(out, lab, nn, rows) for nn in (2, 10, 100)},
                "stress": E, "finite": finite}

    q32 = quality()
    qnx_f32 = q32["qnx"]

    # half-precision gathered positions and the cluster-grouped layout order:
    # same graph, same seed, same step
    variants = {}
    for var in [v for v in args.variants.split(",") if v and v != "none"]:
        fmt, order = (var.split(":") + ["degree"])[:2]
        one_embedding(knn, out, pos_format=fmt, order=order)
        vs, ve = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        vt = []
        for s_ in range(args.steps):
            flush.zero_()
            vs.record(stream)
            one_embedding(knn, out, vk[s_], pos_format=fmt, order=order,
                          after_readback=lambda: ve.record(stream))
            torch.cuda.synchronize()
            vt.append(vs.elapsed_time(ve))
        vms = statistics.mean(vt)
        vkms = statistics.mean(a.elapsed_time(b) for a, b in vk)
        qv = quality(fmt, order)
        variants[var] = {"value": terms * n_iter / (vms / 1e3), "s_to_embed": vms / 1e3,
                         "launch_us": 1e3 * vkms / n_iter, "qnx": qv["qnx"], "cf": qv["cf"],
                         "stress": qv["stress"], "finite": qv["finite"],
                         "qnx_minus_f32": qv["qnx"] - qnx_f32,
                         "equal_precision": abs(qv["qnx"] - qnx_f32) <= 0.01}

    # e2e through the public API from pinned host memory
    e2e = None
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(1, args.steps)
    knn_host = torch.empty((w.M, w.k), dtype=torch.int32, pin_memory=True)
    knn_host.copy_(knn)
    out_host = torch.empty((w.M, 2), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        stamp = []

        def done():
            torch.cuda.synchronize()
            stamp.append(time.perf_counter())

        t = time.perf_counter()
        one_embedding(knn_host, out_host, after_readback=done)
        torch.cuda.synchronize()
        e2e_t.append(stamp[0] - t)
    e2e = {"value": terms * n_iter / statistics.mean(e2e_t) * world, "unit": UNIT,
           "h2d_bytes_per_step": int(knn_host.numel() * 4),
           "d2h_bytes_per_step": int(out_host.numel() * 4), "steps": e2e_steps}

    # roofline of the fused step kernel (algorithmic bytes per launch)
    M = w.M
    nnz = info["nnz_sym"]
    n_slices = (M - info["n_hub"] + 31) // 32
    # per vertex: y, v read + y', v' written (Adadelta: + E[dx^2] read and written)
    state_bytes = 48 if args.opt == "adadelta" else 32
    alg_bytes = state_bytes * M + 4 * nnz + 8 * n_slices + 4 * (info["n_hub"] + 1)
    launch_s = kms / 1e3 / n_iter
    achieved = alg_bytes / launch_s / 1e9
    peaks = measured_peaks()
    tr = step_kernel_traffic()
    gpeak = ivhd.probe_gather(M, 16_777_216, 20)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "peak_source": peaks["source"], "kernel": f"k_step<{args.opt}>",
                "algorithmic_bytes_per_launch": alg_bytes,
                "launch_us": launch_s * 1e6,
                "l2_gather": {
                    "achieved": nnz / launch_s, "peak": gpeak, "unit": "gathers/s",
                    "frac": (nnz / launch_s) / gpeak,
                    "peak_source": "ivhd_probe_gather on this GPU: uniformly random float2 "
                                   f"gathers from {M} elements, indices in registers"}}
    # the binding limit: t_min = max(HBM bytes / HBM peak, gathers / measured gather rate)
    t_hbm = alg_bytes / (peaks["hbm_gbs"] * 1e9)
    t_gather = nnz / gpeak
    roofline["binding"] = {
        "bound": "l2_gather" if t_gather >= t_hbm else "hbm",
        "t_min_us": 1e6 * max(t_hbm, t_gather), "t_hbm_us": 1e6 * t_hbm,
        "t_gather_us": 1e6 * t_gather, "frac": max(t_hbm, t_gather) / launch_s,
        "what": "launch time against the larger of the two lower bounds: the streamed "
                "bytes at the HBM copy peak, and the gathered entries at the measured "
                "random-gather rate (each gather is one 32-byte L2 sector request)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(w, n_iter, args.opt),
                   "parallelism": "replicas" if world > 1 else "single"},
        "s_to_embed": ms / 1e3,
        "kernel_edge_updates_per_s": terms * n_iter / (kms / 1e3),
        "terms": terms, "nnz_sym": nnz, "n_hub": info["n_hub"], "max_degree": info["max_degree"],
        "knn_build_s_untimed": knn_seconds,
        "qnx": {"value": qnx_f32, "k": w.k, "rows": int(rows.numel()),
                "what": "Q_NX(k) of the final embedding on sampled rows (input kNN edges recovered)"},
        "quality_f32": q32,
        "variants": variants,
        "wall_s_timed_region": wall,
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(run_extras(args, dev, stream, flush, local_rank))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nt = host_threads()
        o = oracle_sample(w, args.cpu_seconds, opt=args.opt, threads=nt)
        ser = o["serial"]
        line["cpu_baseline"] = {
            "value": ser["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{ser['iters']} of {n_iter} {args.opt} iterations (FP64, single thread) "
                      f"on a {w.M} x {w.k} kNN-shaped graph with r={w.r} ({o['terms']} terms), "
                      f"{ser['seconds']:.1f} s"}
        if "threads" in o:
            th = o["threads"]
            line["cpu_baseline"]["all_cores"] = {
                "value": th["value"], "unit": UNIT, "cores": th["cores"], "kind": "oracle",
                "sample": f"{th['iters']} iterations of the same loop on {th['cores']} host "
                          f"threads (per-thread force sums added in thread order), "
                          f"{th['seconds']:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# -------------------------------------------------- the other workloads


def config_subline(name: str, opts, dev, stream, flush, steps: int, warmup: int,
                   gpu_index: int) -> dict:
    """One smaller workload timed like the headline: per optimiser, whole embeddings
    (create + n_iter steps + read-back) with CUDA events, the kernel time per
    iteration against the measured random-gather bound, and the quality of the
    result (Q_NX over every vertex up to 1e5 vertices, cf_2/10/100, stress)."""
    import torch

    from paper_2303_05455_gb300 import ivhd

    w = synth.WORKLOADS[name]
    X, labels = synth.workload_features(w)
    knn = ivhd.knn_build(torch.from_numpy(X).to(dev), w.k)
    rows = (torch.arange(w.M, dtype=torch.int64, device=dev) if w.M <= 100_000 else
            torch.from_numpy(synth.sample_rows(w.M, 10_000, 12345)).to(dev))
    lab = torch.from_numpy(labels).to(dev)
    out_buf = torch.empty((w.M, 2), dtype=torch.float32, device=dev)
    gpeak = ivhd.probe_gather(w.M, 16_777_216, 10)
    res = {"config": workload_config(w, w.n_iter)}
    for opt in opts:
        def one(evs=None, end_ev=None):
            emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=opt, a=w.a, b=w.b, seed=w.seed,
                                 stream=stream, device=dev)
            if evs is not None:
                evs[0].record(stream)
            emb.step(w.n_iter)
            if evs is not None:
                evs[1].record(stream)
            emb.positions(out=out_buf)
            if end_ev is not None:
                end_ev.record(stream)  # the embedding is complete; teardown follows
            inf = emb.info()
            try:
                E = emb.stress() if evs is None else None
            except ivhd.IvhdError:
                E = float("nan")
            emb.close()
            return inf, E

        for _ in range(warmup):
            one()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        clocks = ClockSampler(gpu_index)
        torch.cuda.synchronize()
        launches = 0
        for s_ in range(steps):
            flush.zero_()
            ev[s_][0].record(stream)
            inf, _ = one((ev[s_][2], ev[s_][3]), ev[s_][1])
            launches += inf["setup_launches"] + inf["kernel_launches"] + inf["aux_launches"]
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
        kms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
        inf, E = one()
        launch_s = kms / 1e3 / w.n_iter
        t_gather = inf["nnz_sym"] / gpeak
        form = ["one step kernel per step", "one block per call", "8-block cluster per call",
                "persistent grid per call"][inf["launch_form"]]
        if inf["launch_form"] in (1, 2):
            # positions live in shared memory: no L2 gathers to bound the step
            binding = {"bound": "launch form", "launch_form": form, "frac": None,
                       "what": "all steps of a call run in one launch with the positions in "
                               "shared memory; the random-gather bound does not apply"}
        else:
            binding = {"bound": "l2_gather", "launch_form": form, "t_min_us": 1e6 * t_gather,
                       "frac": t_gather / launch_s, "gather_peak": gpeak,
                       "what": "kernel time per iteration against the row entries at the "
                               "measured random-gather rate (ivhd_probe_gather, same size)"}
            if inf["launch_form"] == 0:
                # the chained launches alone, with this step grid (ivhd_probe_launch)
                binding["step_blocks"] = inf["step_blocks"]
                binding["launch_floor_us"] = ivhd.probe_launch(inf["step_blocks"],
                                                               inf["step_threads"], 2000)
        qnx = ivhd.eval_qnx(out_buf, knn, rows)
        res[opt] = {
            "value": inf["n_terms"] * w.n_iter / (ms / 1e3), "unit": UNIT, "s_to_embed": ms / 1e3,
            "steps": steps, "warmup": warmup, "launch_us": 1e6 * launch_s, "binding": binding,
            "quality": {"qnx": qnx, "rows": int(rows.numel()),
                        "cf": {str(nn): ivhd.eval_cf(out_buf, lab, nn, rows) for nn in (2, 10, 100)},
                        "stress": E},
            "terms": inf["n_terms"], "nnz_sym": inf["nnz_sym"], "gpu_launches": launches,
            "clocks": clk}
        if opt == "momentum":
            # half-precision gathered positions, same graph and seed, against this FP32 run
            half = {}
            for fmt in ("f16", "bf16"):
                emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=opt, a=w.a, b=w.b, seed=w.seed,
                                     stream=stream, device=dev, pos_format=fmt)
                emb.step(w.n_iter)
                emb.positions(out=out_buf)
                try:
                    Eh = emb.stress()
                except ivhd.IvhdError:
                    Eh = float("nan")
                emb.close()
                qh = ivhd.eval_qnx(out_buf, knn, rows)
                half[fmt] = {"qnx": qh, "qnx_minus_f32": qh - qnx, "stress": Eh,
                             "stress_rel_to_f32": (Eh - E) / E if E else None,
                             "equal_precision": abs(qh - qnx) <= 0.01}
            res[opt]["half_precision"] = half
    return res


def run_extras(args, dev, stream, flush, gpu_index: int) -> dict:
    from paper_2303_05455_gb300 import bench_batch, bench_warmstart

    out = {"configs": {
        "gmm2k": config_subline("gmm2k", ["momentum"], dev, stream, flush, 5, 3, gpu_index),
        "mnist70k": config_subline("mnist70k", ["momentum", "adadelta"], dev, stream, flush, 5, 3,
                                   gpu_index)}}
    clocks = ClockSampler(gpu_index)
    out["batch64"] = bench_batch.measure()
    out["batch64"]["clocks"] = clocks.stop()
    clocks = ClockSampler(gpu_index)
    out["warmstart"] = bench_warmstart.measure()
    out["warmstart"]["clocks"] = clocks.stop()
    return out


# ------------------------------------------------------ kernel capture modes


def run_capture(args):
    """One kernel family alone, for timing and ncu captures (CUDA-event times as JSON)."""
    import torch

    from paper_2303_05455_gb300 import ivhd

    s = torch.cuda.current_stream()

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    if args.kernel == "step":
        w = synth.WORKLOADS[args.workload]
        if args.graph == "knn":
            X, _ = synth.workload_features(w)
            knn = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k)
            del X
        else:
            knn = torch.from_numpy(synth.random_knn_graph(
                w.M, w.k, w.seed + 1, hub_frac=0.02, n_hubs=max(w.k + 1, w.M // 1000))).cuda()
        torch.cuda.synchronize()
        combos = [(o, f, sh) for o in args.order.split(",") for f in args.pos_format.split(",")
                  for sh in args.shapes_step.split(",")]
        forms = {"auto": None, "multi": False, "grid": "grid", "cluster": "cluster",
                 "block": True}
        for order, fmt, shape in combos:
            parts = shape.split(":")
            hub, vpw, block = (int(v) for v in parts[:3])
            resident = forms[parts[3]] if len(parts) > 3 else None
            for rep in range(args.reps):
                t0 = time.perf_counter()
                emb = ivhd.Embedding(knn, r=w.r, c=w.c, opt=args.opt, a=w.a, b=w.b,
                                     seed=w.seed, pos_format=fmt, order=order,
                                     hub_threshold=hub, vertices_per_warp=vpw,
                                     block_size=block, resident=resident)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                e0, e1 = events()
                e0.record(s)
                emb.step(args.iters)
                e1.record(s)
                torch.cuda.synchronize()
                info = emb.info()
                emb.close()
                print(json.dumps({"workload": w.name, "opt": args.opt, "order": order,
                                  "pos_format": fmt, "shape": shape, "rep": rep,
                                  "create_ms": 1e3 * (t1 - t0),
                                  "us_per_step": 1e3 * e0.elapsed_time(e1) / args.iters,
                                  "n_hub": info["n_hub"], "nnz_sym": info["nnz_sym"],
                                  "max_degree": info["max_degree"],
                                  "launch_form": info["launch_form"]}), flush=True)
    elif args.kernel == "knn":
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
            _, st = ivhd.knn_build(Xd, 5, return_stats=True)
            dt = time.perf_counter() - t0
            print(json.dumps({"rep": rep, "seconds": dt,
                              "tflops": 2.0 * args.M ** 2 * K / dt / 1e12, **st}), flush=True)
    elif args.kernel == "gemm":
        res = []
        for sh in args.shapes.split(","):
            M, N, K = (int(v) for v in sh.split("x"))
            g = torch.Generator(device="cuda").manual_seed(M + N + K)
            A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
            B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
            C = ivhd.gemm_bf16_tn(A, B)
            e0, e1 = events()
            e0.record(s)
            for _ in range(args.reps):
                ivhd.gemm_bf16_tn(A, B, out=C)
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.reps
            ref = A[:64].float() @ B.float().T
            res.append({"M": M, "N": N, "K": K, "ms_per_call": ms,
                        "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12,
                        "max_rel_err_rows0_63": float((C[:64] - ref).abs().max() / ref.abs().max())})
        print(json.dumps(res), flush=True)
    elif args.kernel == "mlp":
        B = args.batch
        net = ivhd.MLP(784, 512, max_batch=B)
        net.init_params(0)
        g = torch.Generator(device="cuda").manual_seed(0)
        X = torch.randint(0, 256, (B * 4, 784), dtype=torch.uint8, device="cuda", generator=g)
        T = torch.randn((B * 4, 2), device="cuda", generator=g)
        for _ in range(3):
            net.train_step(X[:B], T[:B], lr=1e-3, x_scale=1 / 255)
        torch.cuda.synchronize()
        e0, e1 = events()
        t = time.perf_counter()
        e0.record(s)
        for i in range(args.iters):
            b = (i % 4) * B
            net.train_step(X[b:b + B], T[b:b + B], lr=1e-3, x_scale=1 / 255)
        e1.record(s)
        host = time.perf_counter() - t
        torch.cuda.synchronize()
        f0, f1 = events()
        f0.record(s)
        net.forward(X, x_scale=1 / 255)
        f1.record(s)
        torch.cuda.synchronize()
        print(json.dumps({"steps": args.iters, "gpu_ms_per_step": e0.elapsed_time(e1) / args.iters,
                          "host_ms_per_step_enqueue": 1e3 * host / args.iters,
                          "forward_rows": 4 * B, "forward_ms": f0.elapsed_time(f1)}), flush=True)
        net.close()
    elif args.kernel == "resident":
        w = synth.WORKLOADS["gmm2k"]
        X, _ = synth.workload_features(w)
        knn = ivhd.knn_build(torch.from_numpy(X).cuda(), w.k)
        for rep in range(args.reps):
            out = {"rep": rep}
            for resident in (True, "cluster", False):
                emb = ivhd.Embedding(knn, r=w.r, c=w.c, a=w.a, b=w.b, seed=w.seed, opt=args.opt,
                                     resident=resident)
                emb.step(16)
                e0, e1 = events()
                e0.record(s)
                emb.step(args.iters)
                e1.record(s)
                torch.cuda.synchronize()
                key = {True: "resident_us", "cluster": "cluster_us", False: "multi_launch_us"}
                out[key[resident]] = 1e3 * e0.elapsed_time(e1) / args.iters
                emb.close()
            print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return run_capture(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
