"""Cone-energy observable with a hand-written adjoint behind torch.autograd.

    J = sum over cells in a cone (apex at the jet start, axis along the jet,
        half angle 30 deg, radius 3 fm) of E dx^3 after N RK3 steps

as a differentiable function of the initial energy density e(x) and of k_rad,
k_coll of Eq. 3.  The forward pass runs the CUDA step in the precision of the
configuration (FP64, or mixed) keeping a checkpoint every k steps; the
backward pass calls the library's reverse-mode kernels
(hydro_adjoint_backward), which recompute each segment from its checkpoint.  No autograd tape is recorded inside: torch only carries the
inputs and the gradients.
"""
from __future__ import annotations

import torch

from . import hydro as hy


class ConeEnergyRun:
    """Fixed parts of the problem: grid, steps, checkpoint interval, cone, jets,
    and the initial u^i and n fields (the differentiable inputs are e, k_rad, k_coll)."""

    def __init__(self, cfg, nsteps: int, checkpoint_every: int, jets, u_and_n: torch.Tensor, apex, axis,
                 half_angle_deg: float = 30.0, rmax: float = 3.0):
        self.cfg = cfg
        self.shape = (cfg.nz, cfg.ny, cfg.nx)
        self.adj = hy.hydro_adjoint_create(cfg, nsteps, checkpoint_every, apex, axis, half_angle_deg, rmax)
        for j in jets:
            hy.hydro_adjoint_add_jet(self.adj, j.x0, j.direction, j.t_start)
        assert u_and_n.shape == (4,) + self.shape and u_and_n.dtype == torch.float64 and u_and_n.is_cuda
        self.u_and_n = u_and_n.contiguous()

    def prim(self, e: torch.Tensor) -> torch.Tensor:
        return torch.cat([e.reshape((1,) + self.shape), self.u_and_n], 0).contiguous()


class ConeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, e, k_rad, k_coll, run: ConeEnergyRun):
        hy.hydro_adjoint_set_params(run.adj, float(k_rad), float(k_coll))
        J = hy.hydro_adjoint_forward(run.adj, run.prim(e.detach()))
        ctx.run = run
        return torch.tensor(J, dtype=torch.float64, device=e.device)

    @staticmethod
    def backward(ctx, gJ):
        run = ctx.run
        grad_e = torch.empty(run.shape, dtype=torch.float64, device=gJ.device)
        gr, gc = hy.hydro_adjoint_backward(run.adj, float(gJ), grad_e)
        dev = gJ.device
        return grad_e, torch.tensor(gr, dtype=torch.float64, device=dev), \
            torch.tensor(gc, dtype=torch.float64, device=dev), None


def cone_energy(e: torch.Tensor, k_rad: torch.Tensor, k_coll: torch.Tensor, run: ConeEnergyRun) -> torch.Tensor:
    """J(e, k_rad, k_coll); differentiable in all three."""
    return ConeEnergy.apply(e, k_rad, k_coll, run)
