"""Host logic of the benchmark's multi-rank mode (no GPU): N independent
replicas, one per rank, whose job time is the maximum over the ranks and
whose throughput is the sum of their work over that time; the reference arm
runs on rank 0 only.  The ranks are gloo processes on this CPU."""
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


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        job = bench.max_over_ranks(times[rank])
        out[rank] = job
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_maximum_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    port = _free_port()
    times = [0.75, 1.25]
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, port, times, out), nprocs=2, start_method="spawn")
        got = dict(out)
    assert got == {0: 1.25, 1: 1.25}


def test_single_process_time_is_unchanged():
    assert bench.max_over_ranks(0.5) == 0.5


def test_job_throughput_counts_every_replica():
    # two replicas of 10 steps of 1000 updates in 2 s: 10,000 updates/s
    assert bench.job_throughput(1000, 10, 2, 2.0) == pytest.approx(10000.0)
    assert bench.job_throughput(1000, 10, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_json_line(monkeypatch, capsys):
    import json
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.main(["--impl", "reference", "--workload", "rot", "--steps", "1", "--warmup", "3"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["higher_is_better"] is True
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
