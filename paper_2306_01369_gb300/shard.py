"""Sharding of independent environments across GPUs (one process per GPU).

Environments never interact, so the batched workload partitions with no
data-path collective: each rank steps its own subset, and only timing and
metrics are reduced on the host at the end.  A single scene does not shard (a
spatial split would need a halo exchange every projected-Jacobi iteration), so
several GPUs run independent replicas of it.
"""
from __future__ import annotations

import numpy as np


def shard_envs(sizes, world: int):
    """Split environment indices over `world` ranks, balancing the particle total.

    Longest-processing-time greedy: environments in descending size (ties by
    index) go to the currently lightest rank (ties by rank).  Deterministic;
    every environment lands on exactly one rank; each rank's list is ascending.
    """
    sizes = np.asarray(sizes, np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda e: (-int(sizes[e]), e))
    load = [0] * world
    out = [[] for _ in range(world)]
    for e in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(e)
        load[r] += int(sizes[e])
    return [sorted(x) for x in out]


def subset_offsets(env_offsets, envs):
    """Particle index ranges and compacted offsets of a subset of environments."""
    env_offsets = np.asarray(env_offsets, np.int64)
    idx = np.concatenate([np.arange(env_offsets[e], env_offsets[e + 1]) for e in envs]) if envs else \
        np.zeros(0, np.int64)
    sizes = [int(env_offsets[e + 1] - env_offsets[e]) for e in envs]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    return idx, offs
