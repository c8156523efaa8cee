"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2), the max-over-ranks step
time, the whole-job rate built from it, and the reference arm doing no work on ranks other than
0.  (The GPU runs here have one GPU; the same helpers serve torchrun with NCCL.)"""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        ms = bench.max_over_ranks(torch, dist, 1.5 + rank, "cpu")
        q.put((rank, ms, bench.job_rate(3 * 1000, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 2.5  # the slower rank's time, on both ranks
        assert rate == pytest.approx(2 * 3000 / 2.5e-3)


def test_single_process_aggregation_is_the_identity():
    torch = pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(torch, None, 3.25, "cpu") == 3.25
    assert bench.job_rate(100, 1, 2.0) == pytest.approx(5e4)


def test_reference_arm_does_nothing_off_rank_0(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=3, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
