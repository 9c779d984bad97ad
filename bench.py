"""Benchmark of the granular contact step (GranularGym, arxiv 2306.01369) on GB300.

Workload: granular column collapse of 262,144 FP32 spheres (r = 2 mm +-10 %,
40x40-site column at 4.49 mm pitch, released onto a ground plane), mu = 0.6,
dt = 5e-5 s, 20 projected-Jacobi iterations.  One "step" is one time step of the
whole pipeline (binning, sort, contacts, PJA, integration, wrench).  The metric is
particle-steps/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Timing: K time steps after W untimed ones, each bracketed by CUDA events on the
stream the library launches on, with an L2 flush (a 512 MiB write) between timed
steps, outside the events.  The dominant kernel (the PJA sweep) is timed by
events recorded inside the step graph.  Multi-GPU: one process per GPU
(torchrun); each rank steps its own replica of the column (the single-scene
path does not shard), barrier + max over ranks.  End to end ("e2e"): a second
simulation set up the same way steps over the same window through the public API
with host buffers (positions and velocities copied in from pinned memory, stepped,
copied back, every step).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (20 PJA iters)"
UNIT = "particle-steps/s"
WORKLOAD = "column_collapse_262144"
COLLAPSE_STEPS = 2000   # length of the column-collapse run the metric is quoted on


def workload_config(sc, workload="column"):
    base = {"n_particles": sc.n, "pja_iters": sc.params.pja_iters, "dt": sc.params.dt, "mu": sc.params.mu,
            "alpha": sc.params.alpha, "l2": "flushed between timed steps (512 MiB write)"}
    if workload == "excavation":
        return {"workload": "excavation_1048576", **base, "radius_m": "2e-3 +-15%",
                "bed": "128x128x64 sites, settled 3000 steps under the parked scoop",
                "bodies": "container, kinematic scoop on 6 waypoints, 2 free 3 cm cubes"}
    if workload == "batched":
        return {"workload": f"batched_beds_{sc.info.get('envs_total', len(sc.env_offsets) - 1)}", **base,
                "envs": len(sc.env_offsets) - 1,
                "envs_total": sc.info.get("envs_total", len(sc.env_offsets) - 1),
                "bed": "16 layers per environment, settled 1500 steps under the parked tools",
                "bodies": "container + scoop per environment"}
    return {"workload": WORKLOAD, **base, "radius_m": "2e-3 +-10%", "column_sites": "40x40x164",
            "bodies": "ground plane"}


def hash_kw(args):
    """Hash table size: autotuned among 2n, 4n, 8n (results do not depend on it), or the
    fixed factor given on the command line (2: the paper's table size)."""
    return dict(hash_factor=args.hash_factor) if args.hash_factor else dict(hash_tune=1)


def batched_shard(scenes, world, rank, n_steps, n_envs=256):
    """This rank's part of the batched workload: every rank builds the same 256 (or
    n_envs) seeded environments and keeps the subset shard_envs gives it (balanced by
    particle count); the environments never interact, so no collective touches the
    data path."""
    from paper_2306_01369_gb300.shard import shard_scene
    return shard_scene(scenes.batched_beds(n_envs=n_envs, seed=1003, n_steps=n_steps), world, rank)


def setup_workload(args, scenes, gg, rank, stream, world=1):
    """(scene, simulation, untimed steps before the warm-up) of the timed workload."""
    if args.workload == "column":
        sc = scenes.column_collapse(seed=1001 + rank)
        sim = gg.Sim.from_scene(sc, tuning=args.tuning, **hash_kw(args))
        preroll = max(0, (COLLAPSE_STEPS - args.steps) // 2 - args.warmup)
        if preroll:
            sim.step(preroll, stream=stream)
            sim.autotune(stream)          # the collapsing column, not the lattice, decides
        return sc, sim, preroll
    n_run = args.warmup + args.steps + 20
    if args.workload == "excavation":
        sc = scenes.excavation(n=1048576, seed=1002 + rank, n_steps=n_run)
        settle = 3000
    else:
        sc = batched_shard(scenes, world, rank, n_run, args.envs)
        settle = 1500
    parked = scenes.Scene(sc.name, sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params, sc.n_steps,
                          env_offsets=sc.env_offsets, body_offsets=sc.body_offsets)
    sim = gg.Sim.from_scene(parked, tuning=args.tuning, **hash_kw(args))
    sim.step(settle, stream=stream)       # the bed settles, then the tools start digging
    sim.autotune(stream)                  # the settled bed, not the lattice, decides the launch shapes
    bo = sc.body_offsets
    for gb, tw in sc.twist.items():
        if bo is None:
            sim.set_trajectory(gb, tw)
        else:
            e = int(np.searchsorted(bo, gb, side="right") - 1)
            sim.set_trajectory(gb - int(bo[e]), tw, e)
    return sc, sim, settle


# --------------------------------------------------------------------------- #
# distributed plumbing (host logic, covered by gloo tests)
# --------------------------------------------------------------------------- #

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity when world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- #
# clocks during the timed region
# --------------------------------------------------------------------------- #

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- #
# roofline figures of the dominant kernel
# --------------------------------------------------------------------------- #

def pja_bytes(n: int, n_pp: int, n_body: int) -> int:
    """Algorithmic DRAM bytes of one k_pja launch (each array read or written once):
    per particle: velocity estimate in 16 + velocity (base) 16 + counts 4 + estimate out 16;
    per particle-particle contact: partner 4 + normal/psi 16 + impulse in 12 + out 12;
    per particle-body contact: body 4 + normal/psi 16 + contact point 16 + impulse 24."""
    return 52 * n + 44 * n_pp + 60 * n_body


def contacts_bytes(n: int, n_pp: int, n_body: int, n_h: int) -> int:
    """Algorithmic DRAM bytes of one k_contacts launch: per particle position 16 (read
    once, though the kernel reads its own row from the id-ordered copy and candidates
    from the bucket-ordered one), environment 4, velocity 16, counts out 4, first
    velocity estimate out 16, its id in the sorted slot list 4; the bucket table 4 per
    bucket; per pair contact partner 4 + normal/psi 16 + zeroed impulse 12; per body
    contact body 4 + normal/psi 16 + contact point 16 + zeroed impulse 12."""
    return 60 * n + 4 * n_h + 32 * n_pp + 48 * n_body


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


PROFILE_WORKLOAD = {"column": "column_collapse", "excavation": "excavation", "batched": "batched_beds"}


def stage_kernels(flags):
    """(sweep kernel, contact-stage kernels) that a launch-shape set with GG_TUNE_* names
    `flags` runs."""
    if "detect" in flags:                 # one launch holds the contact stage and the sweeps
        return "k_detect_sweeps", "k_detect_sweeps"
    if "oneloop" in flags:                # every iteration walks the cells again
        sweep = "k_oneloop"
    else:
        sweep = "k_pja_fused" if "fused" in flags else ("k_pja_lean" if "lean" in flags else "k_pja")
    contacts = "k_pairs_half+k_pairs_finish" if "half" in flags else "k_contacts"
    return sweep, contacts


def profile_traffic(kernel: str, workload: str, kernel_digest: str):
    """ncu DRAM bytes per launch of `kernel` (the contact stage's kernels summed) from its
    committed profile summary ("key: value" lines) on this workload, if it was taken on
    the current kernel source (else None)."""
    stem = kernel.split("+")[0]
    if workload not in PROFILE_WORKLOAD:
        return None
    path = os.path.join(ROOT, "profiles", f"{stem}_{PROFILE_WORKLOAD[workload]}.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
    except OSError:
        return None
    if kv.get("kernel_digest") != kernel_digest:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ("gg_kernels.cu", "gg_device.cuh"):
        with open(os.path.join(ROOT, "paper_2306_01369_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------- #
# arms
# --------------------------------------------------------------------------- #

ORACLE_BLOCK = 16384     # spheres of the column's bottom layers the oracle steps
ORACLE_PREROLL = 800     # untimed oracle steps first: the block lands and its contacts form


def column_block(sc, m=ORACLE_BLOCK):
    """The lowest m spheres of the column (its bottom layers: the lattice is z-major),
    as a scene of their own with the same recipe; the oracle's bounded sample."""
    from paper_2306_01369_gb300 import scenes
    return scenes.Scene(f"{sc.name}_bottom{m}", sc.pos_r[:m].copy(), sc.vel[:m].copy(), sc.mass[:m].copy(),
                        sc.bodies, sc.params, sc.n_steps)


def oracle_sample(sc, seconds=15.0, max_steps=4000, threads=None):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload: the
    column's bottom block, advanced ORACLE_PREROLL steps untimed from the generator's
    state (it lands and packs against the ground), then whole steps until `seconds`
    have passed.  Oracle inputs never come from the CUDA path."""
    import oracle
    threads = threads or os.cpu_count() or 1
    blk = column_block(sc)
    o = oracle.Sim(blk.pos_r, blk.vel, blk.mass, blk.bodies, blk.params, n_threads=threads)
    o.step(ORACLE_PREROLL)
    x0, v0 = o.x.copy(), o.v.copy()
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    cbar = o.stats.n_pp / blk.n
    o1 = oracle.Sim(blk.pos_r, blk.vel, blk.mass, blk.bodies, blk.params, n_threads=1)
    o1.set_state(x0, v0)
    t1 = time.perf_counter()
    o1.step(5)
    one = blk.n * 5 / (time.perf_counter() - t1)
    return {"value": blk.n * steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} time steps of the column's bottom {blk.n} spheres (same recipe) after "
                      f"{ORACLE_PREROLL} untimed ones (landed; {cbar:.2f} pair contacts per sphere at the end), "
                      f"FP64 C oracle, {threads} OpenMP threads; {el:.1f} s",
            "single_core_value": one, "single_core_sample": "5 steps of the same block from the same state, 1 thread"}


def _oracle_rate(sc, pos, vel, steps, threads=None):
    """The FP64 oracle's particle-steps/s over `steps` whole steps from (pos, vel)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    o = oracle.Sim(pos, vel, sc.mass, sc.bodies, sc.params, twist=sc.twist, n_threads=threads)
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    return {"value": sc.n * steps / el, "cores": threads,
            "sample": f"{steps} whole steps of {sc.n} spheres, {threads} OpenMP threads, {el:.2f} s"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same metric and workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2306_01369_gb300 import scenes
    import oracle
    oracle.build()
    sc = scenes.column_collapse()
    threads = os.cpu_count() or 1
    # bounded sample per step: the column's bottom block (same recipe), landed first
    # (ORACLE_PREROLL untimed steps), then one oracle time step per step
    blk = column_block(sc)
    m = blk.n
    o = oracle.Sim(blk.pos_r, blk.vel, blk.mass, blk.bodies, blk.params, n_threads=threads)
    o.step(ORACLE_PREROLL)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    el = time.perf_counter() - t0
    v = m * args.steps / el
    cfg = workload_config(sc)
    cfg.update(n_particles=m, sample=f"the column's bottom {m} spheres (of {sc.n}), landed: "
                                     f"{ORACLE_PREROLL} untimed steps before the warm-up")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "contacts_per_particle": o.stats.n_pp / m,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: one FP64 oracle time step of the column's bottom {m} spheres "
                                       f"(same recipe, landed), {threads} OpenMP threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _timed_steps(sim, steps, stream, torch):
    """Device ms of `steps` steps (events on the library's stream)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps, stream=stream)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def steady_backward(gg, torch, dev, stream, s32, ds, p, v, pose, mu, mass, grad_twist, fwd_ms, scoop_mass):
    """The differentiable rollout and its reverse pass on one simulation that is kept (a
    training loop's steady state): from the second pass on, the taped forward and the
    backward reuse the tape, the checkpoints and the per-slot graphs.  Seeds: the
    gradient of the same loss at the autograd rollout's final state."""
    import dataclasses
    pd, posed = p.detach().requires_grad_(), pose.detach().requires_grad_()
    g_pos, g_pose = torch.autograd.grad(scoop_mass(pd, mass, posed, ds.bodies[1].shape12(), ds.info["eps"]),
                                        (pd, posed))
    g_vel = torch.zeros_like(v)          # the loss does not read the velocities
    keep = gg.Sim(s32.pos_r, s32.vel, s32.mass, dataclasses.replace(s32.params, mu=float(mu.detach())))
    try:
        keep.set_bodies(s32.bodies)
        for b, twb in s32.twist.items():
            keep.set_trajectory(b, twb)
        keep.tape_reserve(200, 20)
        st0 = keep.state()
        steady = []
        for _ in range(3):
            keep.set_state(st0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            keep.step_taped(1, 200, stream=stream)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            dtw, dmu = keep.backward(g_pos, g_vel, g_pose, stream=stream)
            torch.cuda.synchronize(dev)
            t2 = time.perf_counter()
            steady.append((1e3 * (t1 - t0), 1e3 * (t2 - t1)))
    finally:
        keep.close()
    return {"steady_taped_forward_ms": steady[-1][0], "steady_backward_ms": steady[-1][1],
            "steady_bwd_over_fwd": steady[-1][1] / fwd_ms,
            "steady_grad_equals_autograd": bool(torch.equal(dtw.reshape(grad_twist.shape), grad_twist)),
            "steady_note": "third taped forward + backward on one kept simulation, set back to the start "
                           f"state each time; the first pass measured {steady[0][0]:.1f} + {steady[0][1]:.1f} ms"}


def extras(torch, dev, stream, steps_batched=50, steps_exc=100, seconds_cap=180.0, settle_steps=1500,
           settle_steps_exc=3000):
    """The other figures of the headline metric, one GPU: batched env-steps/s against
    a loop of the plain single-environment path, backward/forward time of the
    differentiable workload, and the 1M-sphere excavation throughput."""
    from paper_2306_01369_gb300 import gg, scenes
    from paper_2306_01369_gb300.autograd import rollout, scoop_mass
    out = {}
    t_start = time.perf_counter()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the column's pile: 262,144 spheres run for 20,000 steps (1 s; the collapse is still
    # creeping then), repose angle and centre of mass of what it has become; then the
    # throughput and rooflines of 200 steps of that densely packed pile
    from paper_2306_01369_gb300.stats import pile_statistics
    col = scenes.column_collapse()
    sim = gg.Sim.from_scene(col, hash_tune=1)
    sim.step(20000, stream=stream)
    sim.sync(stream)
    pv = sim.pos_vel()
    ke = 0.5 * float((col.mass * (pv[1].astype(np.float64) ** 2).sum(1)).sum())
    angle, com, nbins = pile_statistics(pv[0][:, :3], col.mass, float(col.pos_r[:, 3].max()))
    sim.autotune(stream)                  # the packed pile, not the lattice, decides
    for w in range(4):
        sim.enable_timing(w % 2 == 1)
        sim.step(1, stream=stream)
    md = measure(sim, col, 200, stream, torch, flush, workload="column_pile")
    dense = {"particle_steps_per_s": col.n * 200 / (md["total_ms"] * 1e-3), "ms_per_step": md["total_ms"] / 200,
             "contacts_per_particle": md["contacts_per_particle"], "tuning_set": sim.tuning_selected,
             "hash_table": f"n_h = {sim.hash_size(0) / col.n:.0f} n", "roofline": md["roofline"],
             "roofline_next": md["roofline_next"], "timed_steps": [20004, 20204]}
    sim.close()
    out["column_pile"] = {"workload": "column collapse 262,144, mu 0.6, after 20,000 steps (1 s)",
                          "repose_angle_deg": angle, "centre_of_mass_m": [float(c) for c in com],
                          "initial_height_m": float(col.pos_r[:, 2].max()), "fit_bins": nbins,
                          "kinetic_energy_j": ke, "dense_steps": dense}
    # small settle: 4,096 spheres in an open box, 200 steps (the oracle runs it whole)
    ss = scenes.settle_box(n=4096, n_steps=200)
    sim = gg.Sim.from_scene(ss, hash_tune=1)
    sim.step(3, stream=stream)
    sim.set_particles(ss.pos_r, ss.vel, stream=stream)
    ms = _timed_steps(sim, 200, stream, torch)
    sim.sync(stream)
    sim.close()
    orc = _oracle_rate(ss, ss.pos_r, ss.vel, 200)
    out["small_settle"] = {"workload": "4,096 spheres settling in a 0.2 m open box, 200 steps, I=20",
                           "particle_steps_per_s": ss.n * 200 / (ms * 1e-3), "ms_per_step": ms / 200,
                           "oracle_particle_steps_per_s": orc["value"], "oracle_threads": orc["cores"],
                           "oracle_sample": orc["sample"]}
    # batched: 256 environments, 8k-64k spheres each; the beds settle (tools parked
    # above them) before the tools start digging and the timing starts
    sc = scenes.batched_beds(n_envs=256, n_steps=steps_batched + 10)
    parked = scenes.Scene(sc.name, sc.pos_r, sc.vel, sc.mass, sc.bodies, sc.params, sc.n_steps,
                          env_offsets=sc.env_offsets, body_offsets=sc.body_offsets)
    sim = gg.Sim.from_scene(parked, hash_tune=1)
    sim.step(settle_steps, stream=stream)
    sim.autotune(stream)
    bo = sc.body_offsets
    for gb, tw in sc.twist.items():
        e = int(np.searchsorted(bo, gb, side="right") - 1)
        sim.set_trajectory(gb - int(bo[e]), tw, e)
    sim.step(3, stream=stream)
    settled_pos, settled_vel = sim.pos(), sim.vel()
    ms = _timed_steps(sim, steps_batched, stream, torch)
    sim.sync(stream)
    st = sim.stats()
    E = len(sc.env_offsets) - 1
    batched = E * steps_batched / (ms * 1e-3)
    kps = sim.kernels_per_step
    sim.close()
    # the same environments from the same settled state, each stepped alone (a sample
    # of 16, scaled to all 256)
    per_env_ms, sample = [], list(range(0, E, E // 16))[:16]
    for e in sample:
        o0, o1 = int(sc.env_offsets[e]), int(sc.env_offsets[e + 1])
        b0, b1 = int(sc.body_offsets[e]), int(sc.body_offsets[e + 1])
        es = scenes.Scene("env", settled_pos[o0:o1], settled_vel[o0:o1], sc.mass[o0:o1], sc.bodies[b0:b1],
                          sc.params, sc.n_steps,
                          twist={gb - b0: t[3:] for gb, t in sc.twist.items() if b0 <= gb < b1})
        one = gg.Sim.from_scene(es, hash_tune=1)
        one.step(3, stream=stream)
        per_env_ms.append(_timed_steps(one, 20, stream, torch) / 20)
        one.close()
    loop = 1.0 / (statistics.mean(per_env_ms) * 1e-3)
    out["batched"] = {"workload": f"{E} environments, {sc.n} spheres (8k-64k each), I=20, beds settled for "
                                  f"{settle_steps} steps before the tools dig", "env_steps_per_s": batched,
                      "particle_steps_per_s": sc.n * steps_batched / (ms * 1e-3),
                      "mean_pp_per_particle": st["n_pp"] / sc.n,
                      "loop_of_plain_env_steps_per_s": loop, "speedup_vs_loop": batched / loop,
                      "timed_steps": steps_batched, "kernels_per_step": kps,
                      "loop_sample": f"{len(sample)} of {E} environments stepped alone, 20 steps each"}
    # differentiable: 32,768 spheres, 200 steps, checkpoint every 20
    if time.perf_counter() - t_start < seconds_cap:
        ds = scenes.diff_scene(n=32768, n_steps=200)
        settle = gg.Sim(ds.pos_r, ds.vel, ds.mass, ds.params)
        settle.set_bodies(ds.bodies)
        settle.step(600, stream=stream)
        pos, vel = settle.pos(), settle.vel()
        settle.close()
        s32 = scenes.Scene("diff32k", pos, vel, ds.mass, ds.bodies, ds.params, 200, twist=ds.twist, info=ds.info)
        plain = gg.Sim.from_scene(s32)
        plain.step(2, stream=stream)
        plain.set_particles(pos, vel, stream=stream)
        fwd_ms = _timed_steps(plain, 200, stream, torch)
        plain.close()
        mass = torch.tensor(ds.mass, device=dev)
        for _ in range(2):   # the first pass is untimed: torch JIT-compiles the loss kernels on first use
            tw = torch.tensor(ds.twist[1], device=dev, requires_grad=True)
            mu = torch.tensor(float(ds.params.mu), device=dev, requires_grad=True)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            p, v, pose = rollout(tw, mu, s32, 1, 20)
            L = scoop_mass(p, mass, pose, ds.bodies[1].shape12(), ds.info["eps"])
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            L.backward()
            torch.cuda.synchronize(dev)
            t2 = time.perf_counter()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        tw = torch.tensor(ds.twist[1], device=dev, requires_grad=True)
        mu = torch.tensor(float(ds.params.mu), device=dev, requires_grad=True)
        p, v, pose = rollout(tw, mu, s32, 1, 20)
        L = scoop_mass(p, mass, pose, ds.bodies[1].shape12(), ds.info["eps"])
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        out["differentiable"] = {"workload": "32,768 spheres + scoop, 200 steps, I=20, checkpoint every 20",
                                 "forward_ms": fwd_ms, "taped_forward_ms": 1e3 * (t1 - t0),
                                 "backward_ms": 1e3 * (t2 - t1), "bwd_over_fwd": 1e3 * (t2 - t1) / fwd_ms,
                                 "grad_norm_twist": float(tw.grad.norm()), "dL_dmu": float(mu.grad),
                                 "autograd_note": "each rollout creates, autotunes and tapes a new simulation; "
                                                  "its backward captures every per-slot graph and frees the tape"}
        # the same rollout and reverse pass on one simulation that is kept (a training
        # loop's steady state): from the second pass on, the taped forward and the
        # backward reuse the tape, the checkpoints and the per-slot graphs
        try:
            out["differentiable"].update(steady_backward(gg, torch, dev, stream, s32, ds, p, v, pose, mu, mass,
                                                         tw.grad, fwd_ms, scoop_mass))
        except gg.GGError as e:      # reported in the line; the other figures still run
            out["differentiable"]["steady_error"] = str(e)
    # the gear tower (Sec. III, Fig. helical-gear-benchmark): 65,536 spheres in a tube
    # with a cyclic vertical boundary, n helical gears (GRID bodies sharing one baked
    # grid) on its axis; throughput against the number of gears (the paper's claim:
    # the gridded lookup costs the same whatever the geometry)
    if time.perf_counter() - t_start < seconds_cap:
        gear = scenes.gear_body(10, 0.003, 0.012, margin=0.005)
        rates = {}
        for nb in (0, 5, 10, 20):
            ts = scenes.gear_tower(n=65536, n_gears=nb, gear=gear)
            sim = gg.Sim.from_scene(ts, max_bodies=21)
            sim.step(300, stream=stream)
            ms = _timed_steps(sim, 100, stream, torch)
            sim.sync(stream)
            st = sim.stats()
            rates[str(nb)] = {"particle_steps_per_s": ts.n * 100 / (ms * 1e-3), "ms_per_step": ms / 100,
                              "n_pp": st["n_pp"], "n_body": st["n_body"]}
            sim.close()
        out["gear_tower"] = {"workload": "65,536 spheres in a 6 cm tube with a cyclic vertical boundary and n "
                                         "helical gears (GRID bodies: 10 teeth, module 3 mm, 0.75 mm samples) "
                                         "spinning at U(-4, 4) rad/s, I=20; timed steps 300-400",
                             "by_gear_count": rates, "grid_samples": int(gear.grid.values.size)}
    # depth observations (Sec. III-A): the 72x36 sky camera and the 36x36 ego camera on
    # the settled 1M-sphere excavation bed are timed in the excavation block below
    # ablations of the paper's design choices on the column (262,144 spheres, 1,000
    # steps into the collapse): binning by counting sort vs the paper's per-bucket
    # linked lists (Alg. 2), and the hash table size n_h (Fig. hashtable-benchmark,
    # whose heuristic is n_h = 2n)
    if time.perf_counter() - t_start < seconds_cap:
        col = scenes.column_collapse()
        abl = {}
        for name, kw in (("sort_nh2n", dict(tuning=1, hash_factor=2)), ("lists_nh2n", dict(tuning=7, hash_factor=2)),
                         ("sort_nh1n", dict(tuning=1, hash_factor=1)), ("lists_nh1n", dict(tuning=7, hash_factor=1)),
                         ("sort_nh4n", dict(tuning=1, hash_factor=4)), ("lists_nh4n", dict(tuning=7, hash_factor=4)),
                         ("sort_nh8n", dict(tuning=1, hash_factor=8)), ("lists_nh8n", dict(tuning=7, hash_factor=8))):
            sim = gg.Sim.from_scene(col, **kw)
            sim.step(1000, stream=stream)
            ms = _timed_steps(sim, 100, stream, torch)
            sim.enable_timing(True)
            sim.step(1, stream=stream)
            stg = sim.stage_ms()
            sim.close()
            abl[name] = {"ms_per_step": ms / 100, "binning_us": 1e3 * stg["bin_sort"],
                         "contacts_us": 1e3 * stg["contacts"]}
        out["ablations"] = {"workload": "column collapse 262,144, steps 1000-1100; stage times from one "
                                        "instrumented step after the timed ones", "configs": abl}
        # the hash-table-size experiment at the sizes of Fig. hashtable-benchmark: columns
        # of 1k-65k spheres after 1,000 steps, step time at n_h = 1n .. 8n, both binnings
        curve = {}
        for nc in (1024, 4096, 16384, 65536):
            colc = scenes.column_collapse(n=nc)
            for name, tuning in (("sort", 1), ("lists", 7)):
                row = {}
                for hf in (1, 2, 4, 8):
                    sim = gg.Sim.from_scene(colc, tuning=tuning, hash_factor=hf)
                    sim.step(1000, stream=stream)
                    row[f"nh{hf}n"] = _timed_steps(sim, 200, stream, torch) / 200
                    sim.close()
                curve[f"{name}_n{nc}"] = {"ms_per_step": row,
                                          "speedup_vs_2n": {k: row["nh2n"] / v for k, v in row.items()}}
        out["hashtable_sizes"] = {"workload": "columns of 1,024-65,536 spheres (same recipe), steps 1000-1200, "
                                               "fixed launch shapes (sets 1 and 7)", "configs": curve}
        # the loop-structure experiment (Sec. II-D, Fig. warp-divergence-performance):
        # TwoLoopsSplit (detection, then one launch per sweep), TwoLoopsFused (both loops
        # in one cooperative launch) and OneLoop (every iteration walks the cells again),
        # binning by lists, on columns of 1k-262k spheres 1,000 steps into the collapse
        n_sets = gg.load().gg_tuning_count()
        by_flags = {frozenset(gg.tuning_flags(k)): k for k in range(n_sets, 0, -1)}
        forms = (("TwoLoopsSplit", by_flags[frozenset({"lists"})]),
                 ("TwoLoopsFused", by_flags[frozenset({"lists", "detect"})]),
                 ("OneLoop", by_flags[frozenset({"lists", "oneloop"})]))
        loops = {}
        for nc in (1024, 4096, 16384, 65536, 262144):
            colc = scenes.column_collapse(n=nc)
            row = {}
            for name, tuning in forms:
                sim = gg.Sim.from_scene(colc, tuning=tuning)
                sim.step(1000, stream=stream)
                row[name] = _timed_steps(sim, 100, stream, torch) / 100
                sim.close()
            loops[f"n{nc}"] = {"ms_per_step": row, "time_vs_split": {k: v / row["TwoLoopsSplit"] for k, v in row.items()}}
        out["loop_structure"] = {"workload": "columns of 1,024-262,144 spheres (same recipe), steps 1000-1100, "
                                             "lists binning, n_h = 2n; time_vs_split = the form's step time / the split form's",
                                 "sets": {name: k for name, k in forms}, "configs": loops}
    # excavation: 1,048,576 spheres, scoop, two free cubes, I = 30
    if time.perf_counter() - t_start < seconds_cap:
        ex = scenes.excavation(n=1048576, n_steps=steps_exc + 20)
        parked = scenes.Scene(ex.name, ex.pos_r, ex.vel, ex.mass, ex.bodies, ex.params, ex.n_steps)
        sim = gg.Sim.from_scene(parked, wrench_history=1, hash_tune=1)
        sim.step(settle_steps_exc, stream=stream)   # the bed settles under the parked scoop
        sim.autotune(stream)
        sim.set_trajectory(1, ex.twist[1])
        for w in range(10):
            sim.enable_timing(w % 2 == 1)
            sim.step(1, stream=stream)
        # every step: the step, then its body wrenches (force readback, Sec. III-C) copied
        # into pinned host memory and waited for, as a controller reading forces would
        wr_h = torch.empty(sim.n_envs * sim.max_bodies * 6, dtype=torch.float32).pin_memory()
        me = measure(sim, ex, steps_exc, stream, torch, flush, workload="excavation",
                     readback=lambda k: sim.read("BODY_WRENCH", out=wr_h, stream=stream))
        ms = me["total_ms"]
        sim.sync(stream)
        st = sim.stats()
        # the observations of one step: sky camera over the whole bed, ego camera from the
        # scoop's side looking at the bed (every body traced)
        foot = ex.info["side"] * ex.info["pitch"]
        sky = scenes.Camera(kind=scenes.HEIGHT_CAMERA, width=72, height=36, extent=(foot, 0.5 * foot), empty=0.0)
        ego = scenes.Camera(kind=scenes.DEPTH_CAMERA, width=36, height=36, pos=(-0.45 * foot, 0.0, 0.45),
                            quat=scenes._quat_from_rotvec((0.0, 2.41, 0.0)), fov_y=1.2, near=0.01, far=1.5,
                            march_steps=96, march_eps=1e-4)
        img_s = torch.empty((36, 72), dtype=torch.float32, device=dev)
        img_e = torch.empty((36, 36), dtype=torch.float32, device=dev)
        for _ in range(3):
            sim.render(sky, out=img_s, stream=stream)
            sim.render(ego, out=img_e, stream=stream)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        for _ in range(20):
            sim.render(sky, out=img_s, stream=stream)
        e1.record(stream)
        for _ in range(20):
            sim.render(ego, out=img_e, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        cams = {"sky_72x36_us": 1e3 * e0.elapsed_time(e1) / 20, "ego_36x36_us": 1e3 * e1.elapsed_time(e2) / 20,
                "ego_pixels_hit": int((img_e < 1.5).sum())}
        out["excavation"] = {"workload": f"1,048,576 spheres, scoop + 2 free cubes + container, I=30, bed settled "
                                         f"for {settle_steps_exc} steps before the scoop digs; every timed step "
                                         f"includes its wrench readback to pinned host memory (waited for)",
                             "cameras": cams,
                             "particle_steps_per_s": ex.n * steps_exc / (ms * 1e-3), "ms_per_step": ms / steps_exc,
                             "timed_steps": [10, 10 + steps_exc], "n_pp_last": st["n_pp"], "n_body_last": st["n_body"],
                             "contacts_per_particle": me["contacts_per_particle"], "tuning_set": sim.tuning_selected,
                             "hash_table": f"n_h = {sim.hash_size(0) / ex.n:.0f} n",
                             "roofline": me["roofline"], "roofline_next": me["roofline_next"],
                             "wrench_readback_bytes_per_step": int(wr_h.numel() * 4)}
        sim.close()
        if time.perf_counter() - t_start < seconds_cap:   # the oracle on the generator's (unsettled) bed
            orc = _oracle_rate(ex, ex.pos_r, ex.vel, 2)
            out["excavation"].update({"oracle_particle_steps_per_s": orc["value"], "oracle_threads": orc["cores"],
                                      "oracle_sample": orc["sample"] + ", from the initial lattice bed"})
    return out


SAMPLE_EVERY = 10   # one timed step in ten carries the stage-timing events (they cost ~18 us)


def table_buckets(sim, sc):
    """Buckets of the hash tables in use (sum over environments)."""
    E = len(sc.env_offsets) - 1 if sc.env_offsets is not None else 1
    return sum(sim.hash_size(e) for e in range(E))


def measure(sim, sc, steps, stream, torch, flush, workload="column", readback=None):
    """Time `steps` steps of `sim` (events on the library's stream around each step, the
    L2 flushed between steps outside them); every SAMPLE_EVERY-th step carries the stage
    events, from which the sweep's and the contact stage's live durations and, with the
    step's contact counts, their algorithmic bytes come.  readback(k), if given, runs
    after each step inside its events (a per-step host readback).  Returns step times,
    the roofline of the kernel with the larger share and of the other, and the mean
    number of particle-particle contacts per particle over the sampled steps."""
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    pja_ms, pja_b, con_ms, con_b = 0.0, 0, 0.0, 0
    sampled, cbar, st = [], [], None
    H = table_buckets(sim, sc)
    for k in range(steps):
        inst = k % SAMPLE_EVERY == 0
        sim.enable_timing(inst)                   # selects the step graph (both already captured)
        flush.fill_(float(k))                     # evict L2 between timed steps (outside the events)
        ev0[k].record(stream)
        sim.step(1, stream=stream)
        if readback is not None:
            readback(k)
        ev1[k].record(stream)
        if inst:
            st = sim.stage_ms()                   # waits for this step
            pja_ms += st["pja"]
            con_ms += st["contacts"]
            c = sim.stats()
            pja_b += sc.params.pja_iters * pja_bytes(sc.n, c["n_pp"], c["n_body"])
            con_b += contacts_bytes(sc.n, c["n_pp"], c["n_body"], H)
            cbar.append(c["n_pp"] / sc.n)
            sampled.append(k)
    torch.cuda.synchronize()
    sim.enable_timing(False)
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
    sampled_ms = sum(step_ms[k] for k in sampled)
    peak, peak_kind = measured_peaks()
    digest = kernel_digest()

    def roof(kernel, total_ms, total_bytes, launches):
        avg_s = total_ms * 1e-3 / launches
        per_launch = total_bytes / launches
        achieved = per_launch / avg_s / 1e9
        return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy), burst",
                "traffic": profile_traffic(kernel, workload, digest), "bytes_per_launch": per_launch,
                "avg_launch_us": avg_s * 1e6, "share_of_step": total_ms / sampled_ms,
                "sampled_steps": len(sampled)}

    sweep_kernel, contact_kernels = stage_kernels(sim.tuning_flags)
    if sweep_kernel == contact_kernels:   # detection and sweeps in one launch per step
        roofs = [roof(sweep_kernel, pja_ms + con_ms, pja_b + con_b, len(sampled)), None]
    else:
        sweep_launches = len(sampled) * (1 if sweep_kernel == "k_pja_fused" else sc.params.pja_iters)
        roofs = [roof(sweep_kernel, pja_ms, pja_b, sweep_launches),
                 roof(contact_kernels, con_ms, con_b, len(sampled))]
        roofs.sort(key=lambda r: -r["share_of_step"])
    return {"step_ms": step_ms, "total_ms": sum(step_ms), "roofline": roofs[0], "roofline_next": roofs[1],
            "contacts_per_particle": float(np.mean(cbar)) if cbar else 0.0, "stage_ms_last_sampled_step": st,
            "table_buckets": H}


def run_gpu(args):
    import torch

    from paper_2306_01369_gb300 import _build, gg, scenes

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()

    stream = torch.cuda.current_stream(dev)
    # untimed pre-roll (the column: so that the timed window sits in the middle of the
    # 2000-step collapse; the beds: settling), then the warm-up, which alternates the
    # plain and the instrumented step graphs so that both are captured before timing
    sc, sim, preroll = setup_workload(args, scenes, gg, rank, stream, world)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for w in range(max(args.warmup, 2)):
        sim.enable_timing(w % 2 == 1)
        sim.step(1, stream=stream)
    sim.sync(stream)
    window = [preroll + args.warmup, preroll + args.warmup + args.steps]

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_push("timed")     # lets ncu --nvtx-include "timed/" select the timed steps
    m = measure(sim, sc, args.steps, stream, torch, flush, workload=args.workload)
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    total_ms = max_over_ranks(m["total_ms"], world, dev)
    sim.sync(stream)
    stats = sim.stats()
    value = sum_over_ranks(float(sc.n * args.steps), world, dev) / (total_ms * 1e-3)
    n_envs_rank = len(sc.env_offsets) - 1 if sc.env_offsets is not None else 1
    env_steps = sum_over_ranks(float(n_envs_rank * args.steps), world, dev) / (total_ms * 1e-3)
    roof_main, roof_other, st = m["roofline"], m["roofline_next"], m["stage_ms_last_sampled_step"]

    # end to end through the public API with host buffers: H2D of the state, one
    # step, D2H of the new state, every step; on the same window of the workload as the
    # timed steps (a second simulation set up the same way, from the same inputs)
    tuning_sel, nh0, kps = sim.tuning_selected, sim.hash_size(0), sim.kernels_per_step
    sim.close()
    e2e_steps = min(args.steps, args.e2e_steps or args.steps)
    _, sim, _ = setup_workload(args, scenes, gg, rank, stream, world)
    sim.step(max(args.warmup, 2), stream=stream)
    state_h = torch.empty(7 * sc.n, dtype=torch.float32).pin_memory()   # positions (n, 4), velocities (n, 3)
    sim.read("POS_VEL", out=state_h, stream=stream)
    pos_h, vel_h = state_h[:4 * sc.n].view(sc.n, 4), state_h[4 * sc.n:].view(sc.n, 3)
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):   # gg_step_io: the state in, one step, the new state out, waited for
        sim.step_io(pos_h, vel_h, state_h, stream=stream)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_val = sum_over_ranks(float(sc.n * e2e_steps), world, dev) / e2e_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and sc.env_offsets is None:
        cpu = oracle_sample(sc, seconds=args.cpu_seconds)
    xtra = None
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "column":
        xtra = extras(torch, dev, stream)

    n_env0 = int(sc.env_offsets[1]) if sc.env_offsets is not None else sc.n
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {**workload_config(sc, args.workload),
                           "parallelism": (f"environments sharded over {world} ranks (no data-path collective)"
                                           if sc.env_offsets is not None else f"{world} independent replicas"),
                           "tuning_set": tuning_sel,
                           "hash_table": f"n_h = {nh0 / n_env0:.0f} n per environment "
                                         f"({'fixed' if args.hash_factor else 'autotuned among 2n, 4n, 8n'})",
                           "timed_steps": window},
                "contacts_per_particle": m["contacts_per_particle"],
                "roofline": roof_main, "roofline_next": roof_other, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "steps": e2e_steps, "window": [window[0], window[0] + e2e_steps],
                        "h2d_bytes_per_step": sc.n * (16 + 12), "d2h_bytes_per_step": sc.n * (16 + 12)},
                "env_steps_per_s": env_steps if sc.env_offsets is not None else None,
                "gpu_launches": kps * args.steps, "clocks": clk,
                "stage_ms_last_sampled_step": st,
                "contacts_last_step": {"n_pp": stats["n_pp"], "n_body": stats["n_body"],
                                       "mean_pp_per_particle": stats["n_pp"] / sc.n},
                "extras": xtra}
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gg", "reference"], default="gg")
    ap.add_argument("--tuning", type=int, default=0)
    ap.add_argument("--hash-factor", type=int, default=0,
                    help="fixed n_h = F n per environment (2: the paper's); 0: the autotuner picks 2n, 4n or 8n")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (0: as many as the timed steps, over the same window)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / adjoint / excavation figures")
    ap.add_argument("--envs", type=int, default=256,
                    help="environments of the batched workload (256; fewer only to profile a smaller case)")
    ap.add_argument("--workload", choices=["column", "excavation", "batched"], default="column",
                    help="the timed workload (column: the headline; the others for profiling at sizes that "
                         "do not fit in L2)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
