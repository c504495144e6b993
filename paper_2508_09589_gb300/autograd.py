"""torch.autograd.Function over the C ABI: objective of the space-time solve as a
differentiable function of the design (Sec. 3.3.3 adjoint sensitivities).

forward: st_set_design, st_solve_forward, st_solve_adjoint (which also returns phi);
backward: st_sensitivities, scaled by the incoming gradient.  All arithmetic runs in
libst.so; this module only passes pointers.
"""
from __future__ import annotations

import torch

from .api import Mesh, options, source


class SpaceTimeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, mesh: Mesh, src, opts, objective: str = "compliance", P: int = 20):
        g = gamma.detach().to(dtype=torch.float64).contiguous()
        if g.is_cuda:
            mesh.set_design(g)
        else:
            mesh.set_design(g.numpy())
        mesh.solve_forward(src, opts)
        phi, _ = mesh.solve_adjoint(objective, P, opts=opts)
        ctx.mesh = mesh
        ctx.shape = gamma.shape
        ctx.device = gamma.device
        ctx.dtype = gamma.dtype
        return torch.tensor(phi, dtype=gamma.dtype, device=gamma.device)

    @staticmethod
    def backward(ctx, grad_out):
        mesh = ctx.mesh
        if ctx.device.type == "cuda":
            out = torch.empty(mesh.design_size, dtype=torch.float64, device=ctx.device)
            mesh.sensitivities(out)
        else:
            out = torch.from_numpy(mesh.sensitivities())
        grad = (grad_out.to(torch.float64) * out).reshape(ctx.shape).to(ctx.dtype)
        return grad, None, None, None, None, None


def objective(gamma: torch.Tensor, mesh: Mesh, src=None, opts=None, kind: str = "compliance", P: int = 20):
    """phi(gamma) with d phi / d gamma available through autograd."""
    return SpaceTimeObjective.apply(gamma, mesh, src or source(), opts or options(), kind, P)


class FilterProject(torch.autograd.Function):
    """Physical design gamma_bar = H(F gamma) of Sec. 3.3.2 (PDE filter st_filter, Heaviside
    projection st_heaviside); the backward pass is F (H'(gamma~) * grad), the same filter
    (it is symmetric)."""

    @staticmethod
    def forward(ctx, gamma: torch.Tensor, mesh: Mesh, r_x: float, r_t: float, beta: float, eta: float,
                rtol: float = 1e-12):
        g = gamma.detach().to(dtype=torch.float64).cpu().contiguous().numpy()
        gt, _ = mesh.filter(g, r_x, r_t, rtol)
        gb, dh = mesh.heaviside(gt, beta, eta)
        ctx.mesh, ctx.dh, ctx.args = mesh, dh, (r_x, r_t, rtol)
        ctx.device, ctx.dtype, ctx.shape = gamma.device, gamma.dtype, gamma.shape
        return torch.from_numpy(gb).to(device=gamma.device, dtype=gamma.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        r_x, r_t, rtol = ctx.args
        gin = grad_out.detach().to(torch.float64).cpu().numpy() * ctx.dh
        g, _ = ctx.mesh.filter(gin, r_x, r_t, rtol)
        return (torch.from_numpy(g).reshape(ctx.shape).to(device=ctx.device, dtype=ctx.dtype),
                None, None, None, None, None, None)


def filter_project(gamma: torch.Tensor, mesh: Mesh, r_x: float = 0.0, r_t: float = 0.0, beta: float = 32.0,
                   eta: float = 0.5):
    """gamma_bar = H(F gamma), differentiable (filter radii <= 0: the paper's 2.4 h and 2.4 dt)."""
    return FilterProject.apply(gamma, mesh, r_x, r_t, beta, eta)
