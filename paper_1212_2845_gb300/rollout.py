"""Differentiable rollout: a ``torch.autograd.Function`` over the adjoint
entry points of the C ABI (``vx_rollout_forward`` / ``vx_rollout_backward``).

``rollout(sim, log_E, phase, n_steps)`` returns the per-body centre-of-mass x
travel over ``n_steps`` steps from the simulator's state at call time; its
backward pass runs the hand-written reverse kernels (state recomputed from
checkpoints every ``checkpoint_every`` steps) and returns d/d(log E) and
d/d(phase) per voxel.  The timestep is held at the simulator's current value:
setting log E does not change it inside a rollout (no derivative through the
stability limit, which depends on the stiffest bond).
"""
from __future__ import annotations

import numpy as np
import torch

from . import vx


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_E, phase, sim, n_steps, checkpoint_every, v0):
        dt = sim.dt()
        sim.set_voxel_params(log_E.detach().cpu().numpy().astype(np.float32),
                             phase.detach().cpu().numpy().astype(np.float32))
        sim.set_dt(dt)                      # frozen timestep
        sim.reset(v0)
        loss = sim.rollout_forward(n_steps, checkpoint_every)
        ctx.sim = sim
        ctx.devices = (log_E.device, phase.device)
        return torch.from_numpy(loss).to(log_E.device)

    @staticmethod
    def backward(ctx, g):
        sim = ctx.sim
        dev = torch.device("cuda", torch.cuda.current_device())
        gE = torch.empty(sim.N, dtype=torch.float32, device=dev)
        gP = torch.empty(sim.N, dtype=torch.float32, device=dev)
        sim.rollout_backward(gE, gP, w_body=g.detach().float().cpu().numpy())
        return gE.to(ctx.devices[0]), gP.to(ctx.devices[1]), None, None, None, None


def rollout(sim, log_E, phase, n_steps, checkpoint_every=100, v0=None):
    """Per-body centre-of-mass x travel (float32 tensor [n_bodies]) of an
    n_steps rollout started from reset(v0), differentiable in log_E and phase
    (float tensors [N], canonical voxel order)."""
    return Rollout.apply(log_E, phase, sim, int(n_steps), int(checkpoint_every), v0)
