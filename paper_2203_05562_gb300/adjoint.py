"""Gradients of an objective of the final displacement with respect to the
critical-state slope M, the viscosity eta, the suction and the initial
preconsolidation pressure, through the hand-written adjoint of the step
(``ppm_adjoint_forward`` / ``ppm_adjoint_reverse``).

Example::

    theta = torch.tensor([M, eta, suction, pc0], dtype=torch.float64, requires_grad=True)
    u = ColumnRun.apply(theta, cfg, v0, 200, 20, "mixed")      # (3, n) on the GPU
    J = top_surface_runout(u, cfg)
    J.backward()                                               # theta.grad
"""
from __future__ import annotations

import numpy as np
import torch

from .ppm import Simulation

PARAMS = ("M", "eta", "suction", "pc0")


class ColumnRun(torch.autograd.Function):
    """u_N = run(theta): n_steps explicit steps of one soil column from its
    initial state; backward runs the reverse sweep from checkpoints kept
    every ckpt_every steps, recomputing the steps between them.  bond_tile
    is the bond kernel's threads per point (32, 64, 128, 256)."""

    @staticmethod
    def forward(ctx, theta, cfg, v0, n_steps, ckpt_every, precision="mixed", bond_tile=32):
        vals = theta.detach().cpu().double().numpy()
        run_cfg = dict(cfg)
        for name, val in zip(PARAMS, vals):
            run_cfg[name] = float(val)
        sim = Simulation(run_cfg, precision=precision, use_graph=False, bond_tile=bond_tile)
        if v0 is not None:
            sim.write("v", v0)
        sim.adjoint_forward(int(n_steps), int(ckpt_every))
        u = sim.read("u", device=True).double()
        ctx.sim = sim
        return u

    @staticmethod
    def backward(ctx, grad_u):
        g = ctx.sim.adjoint_reverse(grad_u.detach().double().contiguous())
        ctx.sim = None
        return torch.from_numpy(np.asarray(g)), None, None, None, None, None, None


def top_surface_runout(u: torch.Tensor, cfg: dict) -> torch.Tensor:
    """J = sum over the top lattice layer of u_x^2 + u_y^2."""
    nxy = int(cfg["nx"]) * int(cfg["ny"])
    top = u[:, -nxy:]
    return (top[0] ** 2).sum() + (top[1] ** 2).sum()
