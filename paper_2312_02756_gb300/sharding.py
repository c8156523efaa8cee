"""Sharding of the data-parallel path over ranks (one process per GPU, torch.distributed).

The elementwise kernels (pair masses, boosts, conversions, transformations and their adjoints)
split into contiguous index ranges with no exchange at all: every rank runs the same call on its
own range.  Jagged events split into contiguous event ranges, balanced by particle count; the one
exchange is a single int64 per rank -- its pair total -- gathered so that every rank can place
its pairs in the globally packed pair array (an exclusive scan of the totals over the ranks).
The per-event combinatorics of the jagged form follows the RDataFrame analyses the paper names as
its next target (Sec. 6); the split itself is the data parallelism of Sec. 4.1's kernels.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int):
    """The contiguous index range [lo, hi) of `rank` among `world` ranks for n elements (sizes
    differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_events(offsets, rank: int, world: int):
    """The event range [e_lo, e_hi) of `rank` and its particle range [p_lo, p_hi): contiguous
    events, split where the running particle count crosses rank * total / world (so that ranks
    hold about the same number of particles).  `offsets` is the int64 array of n_events + 1."""
    off = np.asarray(offsets, dtype=np.int64)
    if off.ndim != 1 or off.size < 1 or off[0] != 0 or np.any(np.diff(off) < 0):
        raise ValueError("offsets must be non-decreasing from 0")
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    n_events, total = off.size - 1, int(off[-1])

    def cut(r):
        if r == 0:
            return 0
        if r == world:
            return n_events
        # the first event boundary at or after the particle quantile r * total / world
        return int(np.searchsorted(off, (r * total + world - 1) // world, side="left"))

    e_lo, e_hi = cut(rank), max(cut(rank), cut(rank + 1))
    return e_lo, e_hi, int(off[e_lo]), int(off[e_hi])


def pair_counts(offsets) -> np.ndarray:
    """n (n - 1) / 2 pairs per event."""
    n = np.diff(np.asarray(offsets, dtype=np.int64))
    return n * (n - 1) // 2


def global_pair_base(local_total: int, group=None):
    """(base, grand_total): the number of pairs held by the ranks before this one, and by all of
    them -- one all-gather of one int64 per rank.  Without an initialised process group this is
    the single-rank answer (0, local_total)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, int(local_total)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    mine = torch.tensor([int(local_total)], dtype=torch.int64, device=device)
    allt = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(allt, mine, group=group)
    totals = [int(t.item()) for t in allt]
    return sum(totals[:rank]), sum(totals)


def event_pair_masses_sharded(particles, offsets, group=None, layout=None):
    """This rank's share of the jagged event pair masses: `particles` and `offsets` are the rank's
    own events (offsets from 0, int64 on the GPU).  Returns (pair_offsets, pair_m, event_sums,
    base, grand_total): pair_offsets index the globally packed pair array (the local ones plus
    the pairs of the ranks before this one), pair_m holds this rank's pairs, which occupy
    [base, base + len(pair_m)) of that array."""
    from . import event_pair_masses
    local_total = int(pair_counts(offsets.cpu().numpy()).sum())
    base, grand = global_pair_base(local_total, group)
    po, pm, sums = event_pair_masses(particles, offsets, local_total, layout=layout)
    return po + base, pm, sums, base, grand
