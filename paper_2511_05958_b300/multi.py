"""Series-sharded replicas across ranks (one process per GPU).

Series are independent, so a batch splits across ranks with no exchange on the data path: each
rank runs the engine on its own shard on its own GPU, and the only communication is gathering
the per-series results afterwards (and, for timing, the maximum of the ranks' times).  Shards
are balanced by the scan cost T^2 m of each series (longest-processing-time-first assignment).
"""
from __future__ import annotations

import numpy as np


def shard_by_cost(steps, m, world: int):
    """Indices of the series each rank processes; every series goes to exactly one rank."""
    steps = np.asarray(steps, np.float64)
    m = np.asarray(m, np.float64)
    cost = steps * steps * m
    order = np.argsort(-cost, kind="stable")
    load = np.zeros(world)
    owner = np.empty(len(order), np.int64)
    for s in order:
        r = int(np.argmin(load))
        owner[s] = r
        load[r] += cost[s]
    return [np.nonzero(owner == r)[0] for r in range(world)], load


def sub_batch(samples, offsets, steps, idx):
    """Samples, offsets and steps of the series `idx` (in that order), packed contiguously."""
    offsets = np.asarray(offsets, np.int64)
    parts = [samples[offsets[s]:offsets[s + 1]] for s in idx]
    sub = np.concatenate(parts) if parts else np.zeros(0, samples.dtype)
    lens = np.array([offsets[s + 1] - offsets[s] for s in idx], np.int64)
    sub_off = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(lens, out=sub_off[1:])
    return sub, sub_off, np.asarray(steps, np.int32)[idx]


def gather_rows(local: dict, idx, S_total: int, group=None):
    """Rank 0 receives every rank's per-series rows and scatters them back to global order.

    local: name -> array with one row per series of this rank's shard (in `idx` order).
    Returns the full arrays on rank 0 and None elsewhere.
    """
    import torch.distributed as dist
    world = dist.get_world_size(group)
    payload = (np.asarray(idx), {k: np.asarray(v) for k, v in local.items()})
    parts = [None] * world if dist.get_rank(group) == 0 else None
    dist.gather_object(payload, parts, dst=0, group=group)
    if dist.get_rank(group) != 0:
        return None
    out = {}
    for ids, arrs in parts:
        for k, v in arrs.items():
            if k not in out:
                out[k] = np.zeros((S_total,) + v.shape[1:], v.dtype)
            out[k][ids] = v
    return out


def max_over_ranks(value: float, group=None, device=None) -> float:
    """The slowest rank's time (all-reduce MAX)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
