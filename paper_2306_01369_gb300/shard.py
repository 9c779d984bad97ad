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


def shard_scene(sc, world: int, rank: int):
    """The environments of a batched scene that rank `rank` of `world` steps: the
    shard_envs subset, with its particles, bodies and tool trajectories compacted
    into a batched scene of its own (every rank builds the same full scene from the
    same seed, so the subsets partition it).  A scene without environments is
    returned unchanged (it does not shard)."""
    from . import scenes as S
    if sc.env_offsets is None:
        return sc
    E = len(sc.env_offsets) - 1
    sizes = np.diff(np.asarray(sc.env_offsets, np.int64))
    envs = shard_envs(sizes, world)[rank]
    idx, offs = subset_offsets(sc.env_offsets, envs)
    bo = np.asarray(sc.body_offsets, np.int64)
    bodies, boffs, twist = [], [0], {}
    for e in envs:
        b0, b1 = int(bo[e]), int(bo[e + 1])
        for gb in range(b0, b1):
            if gb in sc.twist:
                twist[len(bodies) + gb - b0] = sc.twist[gb]
        bodies.extend(sc.bodies[b0:b1])
        boffs.append(len(bodies))
    info = dict(sc.info)
    info.update(envs=envs, shard=f"{rank}/{world}", envs_total=E)
    return S.Scene(f"{sc.name}_shard{rank}of{world}", sc.pos_r[idx], sc.vel[idx], sc.mass[idx], bodies, sc.params,
                   sc.n_steps, twist=twist, env_offsets=offs, body_offsets=np.asarray(boffs, np.uint32), info=info)
