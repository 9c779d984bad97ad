"""torch.autograd.Function over libgg's taped forward and hand-written adjoint.

`rollout(twist, mu, scene, tool)` steps a single-environment scene for
len(twist) steps with the tool body following `twist` (float32 (T, 6), world
frame) and friction coefficient `mu`, and returns the final positions, velocities
and tool pose as CUDA tensors.  Its backward calls gg_backward (checkpoint every
`checkpoint_every` steps, recompute in between), which differentiates contact
generation, the projected-Jacobi iterations and the integrator with the contact
and active sets of the forward held fixed.  Differentiation goes beyond the paper
(its Sec. V names it as future work).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import gg


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, twist, mu, scene, tool, checkpoint_every):
        params = dataclasses.replace(scene.params, mu=float(mu.detach().reshape(-1)[0]))
        dev = twist.device
        sim = gg.Sim(scene.pos_r, scene.vel, scene.mass, params)
        sim.set_bodies(scene.bodies)
        for b, tw in scene.twist.items():
            if b != tool:
                sim.set_trajectory(b, tw)
        tw = twist.detach().to(torch.float32).contiguous()
        sim.set_trajectory(tool, tw)
        T = int(tw.shape[0])
        stream = torch.cuda.current_stream(dev)
        sim.tape_reserve(T, checkpoint_every)
        sim.step_taped(tool, T, stream=stream)
        pos4 = torch.empty((sim.n, 4), dtype=torch.float32, device=dev)
        vel = torch.empty((sim.n, 3), dtype=torch.float32, device=dev)
        bst = torch.empty((sim.n_envs * sim.max_bodies, 16), dtype=torch.float32, device=dev)
        sim.read("POS", out=pos4, stream=stream)
        sim.read("VEL", out=vel, stream=stream)
        sim.read("BODY_STATE", out=bst, stream=stream)
        sim.sync(stream)
        ctx.sim = sim
        return pos4[:, :3].contiguous(), vel, bst[tool, 0:7].contiguous()

    @staticmethod
    def backward(ctx, gpos, gvel, gpose):
        dev = gpos.device
        gpos = gpos.contiguous().to(torch.float32)
        gvel = None if gvel is None else gvel.contiguous().to(torch.float32)
        gpose = None if gpose is None else gpose.contiguous().to(torch.float32)
        dtw, dmu = ctx.sim.backward(gpos, gvel, gpose, stream=torch.cuda.current_stream(dev))
        ctx.sim.close()
        return dtw, dmu.reshape(()), None, None, None


def rollout(twist: torch.Tensor, mu: torch.Tensor, scene, tool: int, checkpoint_every: int = 20):
    """Final (positions (n, 3), velocities (n, 3), tool pose (7,)) after len(twist) steps."""
    return _Rollout.apply(twist, mu, scene, tool, checkpoint_every)


def quat_to_matrix(q: torch.Tensor) -> torch.Tensor:
    q = q / torch.linalg.norm(q)
    w, x, y, z = q[0], q[1], q[2], q[3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)])])


def scoop_mass(pos: torch.Tensor, mass: torch.Tensor, pose: torch.Tensor, shape, eps: float) -> torch.Tensor:
    """Smooth particle mass inside the scoop's cavity: sum_i m_i sigmoid(-f_B(y_i) / eps),
    f_B the signed distance to the cavity box B (half extents shape[3:6], centre
    shape[6:9]) in the tool frame, y_i = R^T (x_i - p)."""
    shape = torch.as_tensor(np.asarray(shape, np.float32), device=pos.device)
    R = quat_to_matrix(pose[3:7])
    y = (pos - pose[0:3]) @ R
    z = y - shape[6:9]
    q = torch.abs(z) - shape[3:6]
    m = torch.clamp(q, min=0.0)
    outside = torch.sqrt((m * m).sum(-1) + 1e-30)
    inside = torch.clamp(q.max(-1).values, max=0.0)
    f = outside + inside
    return (mass * torch.sigmoid(-f / eps)).sum()
