"""Splitting a batch of independent systems across ranks (one GPU per rank).

Systems of a batch never interact, so a batched job shards with no exchange on
the data path: every rank builds one context over its share of the systems
(ff_set_systems with that share's sizes, fields and boxes) and steps it; the
per-system observables are gathered once, when the job ends.  This module holds
the host side of that: which rank takes which systems, the rank's slice of the
concatenated arrays, and the gather that puts per-system results back in the
batch's order.
"""
import numpy as np


def partition_systems(sizes, world):
    """Split systems over `world` ranks, balancing particle counts.

    Longest-processing-time rule: systems in order of decreasing size (ties by
    index) go one by one to the rank holding the fewest particles so far (ties
    to the lowest rank).  The largest load exceeds the smallest by at most the
    largest system.  Deterministic, so every rank computes the same split on
    its own.  Returns one ascending index array per rank (possibly empty when
    there are fewer systems than ranks).
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if sizes.ndim != 1 or np.any(sizes < 1):
        raise ValueError("sizes must be a 1-d array of positive counts")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(i)
        load[r] += int(sizes[i])
    return [np.array(sorted(o), dtype=np.int64) for o in owned]


def rank_slice(batch, idx):
    """The systems `idx` of a batch (dict with pos, u, sizes, fields, box_lo, box_hi; pos and u
    concatenated system by system) as a batch of their own, in the order of `idx`."""
    sizes = np.asarray(batch["sizes"], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    idx = np.asarray(idx, dtype=np.int64)
    rows = [np.arange(starts[i], starts[i + 1]) for i in idx]
    rows = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    out = {"pos": batch["pos"][rows], "u": batch["u"][rows], "sizes": sizes[idx],
           "fields": np.asarray(batch["fields"])[idx], "box_lo": np.asarray(batch["box_lo"])[idx],
           "box_hi": np.asarray(batch["box_hi"])[idx]}
    if "sides" in batch:
        out["sides"] = np.asarray(batch["sides"])[idx]
    return out


def gather_system_values(values, idx, nsys, group=None):
    """All-gather per-system rows (`values[k]` belongs to system `idx[k]`) from every rank of
    the default process group and return an (nsys, ...) array in the batch's order.  Every
    system must be owned by exactly one rank."""
    import torch.distributed as dist

    values = np.asarray(values, dtype=np.float64)
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (np.asarray(idx, dtype=np.int64).tolist(), values.tolist()),
                           group=group)
    shape = next((np.asarray(v).shape[1:] for ids, v in parts if ids), ())
    out = np.zeros((nsys,) + shape, dtype=np.float64)
    seen = np.zeros(nsys, dtype=np.int64)
    for ids, vals in parts:
        vals = np.asarray(vals, dtype=np.float64)
        for k, i in enumerate(ids):
            out[i] = vals[k]
            seen[i] += 1
    if np.any(seen != 1):
        raise ValueError("every system must be owned by exactly one rank")
    return out
