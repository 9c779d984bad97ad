"""Multi-process host logic on CPU (gloo, world size 2): the reductions bench.py
uses for max-over-ranks timing and whole-job throughput, and the environment
sharding of the batched workload (no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2306_01369_gb300.shard import shard_envs, subset_offsets


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank "timed" a different duration and processed its own shard
    mine = shard_envs(sizes, world)[rank]
    t = 1.0 + 0.5 * rank
    units = float(sum(sizes[e] for e in mine))
    tmax = bench.max_over_ranks(t, world)
    total = bench.sum_over_ranks(units, world)
    bench.barrier(world)
    q.put((rank, tmax, total, mine))
    dist.destroy_process_group()


def test_gloo_reductions_and_sharding():
    sizes = [9000, 64000, 8200, 31000, 12000, 50000, 8192]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, tmax, total, mine in res:
        assert tmax == 1.5                       # max over ranks
        assert total == float(sum(sizes))        # every particle counted once
    shards = [r[3] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(len(sizes)))


def test_shard_envs_balanced_and_deterministic():
    rng = np.random.default_rng(0)
    sizes = np.rint(np.exp(rng.uniform(np.log(8192), np.log(65536), 256))).astype(int)
    for world in (1, 2, 4, 8):
        sh = shard_envs(sizes, world)
        assert sh == shard_envs(sizes, world)
        flat = sorted(e for s in sh for e in s)
        assert flat == list(range(256))
        loads = [int(sizes[s].sum()) for s in sh]
        assert max(loads) - min(loads) <= sizes.max()
    idx, offs = subset_offsets(np.concatenate([[0], np.cumsum(sizes)]), [3, 1])
    assert offs[-1] == sizes[3] + sizes[1] and idx.size == offs[-1]


def _shard_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2306_01369_gb300 import scenes
    sc = bench.batched_shard(scenes, world, rank, 8)      # what bench.py --workload batched steps on this rank
    total = bench.sum_over_ranks(float(sc.n), world)
    q.put((rank, sc.info["envs"], sc.n, [int(v) for v in sc.env_offsets], len(sc.bodies), sorted(sc.twist),
           total))
    dist.destroy_process_group()


def test_batched_workload_shards_by_environment():
    """bench.py's batched workload on 2 ranks: each rank builds the full seeded batch
    of 256 environments and steps only its shard; the shards partition the 256
    environments, and the particle counts summed over ranks give the batch total."""
    from paper_2306_01369_gb300 import scenes
    full = scenes.batched_beds(n_envs=256, seed=1003, n_steps=8)
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    envs = [e for r in res for e in r[1]]
    assert sorted(envs) == list(range(256))
    assert sum(r[2] for r in res) == full.n
    sizes = np.diff(full.env_offsets.astype(np.int64))
    for rank, mine, n, offs, nbodies, twist_keys, total in res:
        assert total == float(full.n)
        assert np.array_equal(np.diff(offs), sizes[mine])
        assert nbodies == 2 * len(mine) and twist_keys == [2 * k + 1 for k in range(len(mine))]
    loads = [r[2] for r in res]
    assert max(loads) - min(loads) <= sizes.max()


def test_shard_envs_rejects_empty_world():
    with pytest.raises(ValueError):
        shard_envs([1, 2], 0)
