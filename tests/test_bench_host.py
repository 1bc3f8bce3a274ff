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


def test_clock_sampler_parses_samples_and_reasons(tmp_path, monkeypatch):
    # a stand-in for nvidia-smi that prints one CSV sample every 50 ms
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do\n"
                    "echo '0, 1980, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active'\n"
                    "sleep 0.05\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    cs = bench.ClockSampler(0)
    assert cs.lines, "the first sample is awaited before the timed region"
    import time
    time.sleep(0.3)
    r = cs.stop()
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] >= 3


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    r = bench.ClockSampler(0).stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
