"""Host logic of bench.py's multi-process path, run as gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed (r + 1) seconds, its kernel (r + 1) ms, and did 100 (r + 1) units
    res = bench.aggregate_ranks(float(rank + 1), float(rank + 1), 100.0 * (rank + 1), "cpu")
    q.put((rank, res))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_aggregate_is_max_time_and_sum_of_units(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = (float(world), float(world), 100.0 * world * (world + 1) / 2)
    for r in range(world):
        assert got[r] == want


def test_reference_arm_non_zero_rank_exits_without_work(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    ns = argparse.Namespace(impl="reference", workload="gmm2k", n_iter=None, steps=1, warmup=0,
                            gpus=2)
    assert bench.run_reference(ns) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_small_workload(capsys, monkeypatch):
    import argparse
    import json

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    ns = argparse.Namespace(impl="reference", workload="gmm2k", n_iter=50, steps=2, warmup=1,
                            gpus=1, opt="adadelta")
    assert bench.run_reference(ns) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["config"]["optimizer"] == "adadelta"
