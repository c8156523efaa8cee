"""Sharding of the data-parallel path (paper_2312_02756_gb300.sharding) on CPU: index and event
ranges partition the work, and two gloo ranks (world size 2) place their pairs in the globally
packed pair array through one all-gather of the per-rank pair totals -- the same positions a
single process computes."""
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import gvx_synth as syn  # noqa: E402


def test_shard_range_partitions():
    from paper_2312_02756_gb300 import sharding
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            rs = [sharding.shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1


def test_shard_events_partitions_and_balances():
    from paper_2312_02756_gb300 import sharding
    off = syn.jagged_offsets(syn.rng(300), 10_000)
    for world in (1, 2, 3, 8):
        rs = [sharding.shard_events(off, r, world) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == len(off) - 1
        assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
        assert all(p_lo == off[e_lo] and p_hi == off[e_hi] for e_lo, e_hi, p_lo, p_hi in rs)
        parts = [p_hi - p_lo for _, _, p_lo, p_hi in rs]
        assert max(parts) - min(parts) <= 2 * 64  # within two events (n <= 64) of each other
    empty = np.zeros(5, dtype=np.int64)
    assert sum(e_hi - e_lo for e_lo, e_hi, _, _ in (sharding.shard_events(empty, r, 3) for r in range(3))) == 4
    with pytest.raises(ValueError):
        sharding.shard_events(np.array([1, 2]), 0, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2312_02756_gb300 import sharding
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        off = syn.jagged_offsets(syn.rng(301), 5000)
        e_lo, e_hi, _, _ = sharding.shard_events(off, rank, world)
        local = off[e_lo:e_hi + 1] - off[e_lo]
        counts = sharding.pair_counts(local)
        base, grand = sharding.global_pair_base(int(counts.sum()))
        # the local pair offsets the kernel writes, rebased as event_pair_masses_sharded does
        po = base + np.concatenate([[0], np.cumsum(counts)])
        q.put((rank, e_lo, e_hi, po.tolist(), base, grand))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_place_pairs_globally():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    off = syn.jagged_offsets(syn.rng(301), 5000)
    n = np.diff(off)
    want = np.concatenate([[0], np.cumsum(n * (n - 1) // 2)])
    (r0, lo0, hi0, po0, b0, g0), (r1, lo1, hi1, po1, b1, g1) = out
    assert (lo0, hi1, hi0) == (0, len(n), lo1) and b0 == 0
    assert g0 == g1 == want[-1]
    assert np.array_equal(np.array(po0), want[lo0:hi0 + 1])
    assert np.array_equal(np.array(po1), want[lo1:hi1 + 1])
    assert b1 == want[lo1]
