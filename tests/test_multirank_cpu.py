"""World-size-2 checks of bench.py's multi-rank host logic on CPU (gloo).

Each rank embeds its own independent workload (weak scaling, no data-path
collective); the only collective is the max over ranks of the step time.
"""
import argparse
import json
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import bench
import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        r, wsz, local = bench.dist_env()
        local_ms = [12.5, 30.0][rank]
        ms = bench.max_over_ranks(local_ms)
        value = bench.job_throughput(wsz, 100_000, ms)
        seed = bench.rank_seed(0, r)
        w, _, Y, part = bench.make_workload("dc", seed, 3000)
        out.put((r, wsz, local, ms, value, seed, float(Y[:4].sum()), part.p, int(part.ptr[-1]) + len(part.anchors)))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_max_time_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, ms0, v0, s0, y0, p0, n0), (r1, w1, l1, ms1, v1, s1, y1, p1, n1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert ms0 == ms1 == 30.0                          # slowest rank sets the step time
    assert v0 == v1 == pytest.approx(2 * 100_000 / 0.030)
    assert s0 != s1 and y0 != y1                       # independent workloads per rank
    assert n0 == n1 == 3000                            # own points + anchors: same size per rank


def test_single_process_is_identity():
    assert not tdist.is_initialized()
    assert bench.max_over_ranks(7.25) == 7.25
    assert bench.job_throughput(1, 1000, 10.0) == pytest.approx(1e5)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    ns = argparse.Namespace(workload="dc", seed=0, n=0, warmup=1, steps=1, cpu_parts=1, gpus=2)
    bench.reference_arm(ns)
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_line(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    ns = argparse.Namespace(workload="dc", seed=0, n=3000, warmup=1, steps=1, cpu_parts=1, gpus=1)
    bench.reference_arm(ns)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "points/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
