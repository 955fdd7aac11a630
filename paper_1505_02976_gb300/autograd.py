"""PyTorch autograd interface to the discrete adjoint (``lbm_adjoint``).

``wall_nusselt(eps_field, T_walls, problem, steps)`` returns the mean
Nusselt number on one wall (default the hot W wall) after ``steps`` steps as
a differentiable scalar of the porosity field and of the Dirichlet
temperatures of the W and E walls, ``T_walls = (T_W, T_E)`` whatever wall the
loss is taken on (both must be Dirichlet walls of the problem).

``forward`` only advances the lattice and reads the Nusselt number.
``backward`` runs ``lbm_adjoint`` from the same initial state: the forward
steps again with checkpoints every ceil(sqrt(steps)) steps, then the adjoint
of every step back to step 0 with the states recomputed from the
checkpoints; nothing of the adjoint runs unless a gradient is requested.
The loss is returned on the device of ``eps_field``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


def _lattice(eps_field, T_walls, problem, precision):
    p = dict(problem)
    if p["bc"][0] != "dirichlet" or p["bc"][1] != "dirichlet":
        raise ValueError("T_walls are the W and E Dirichlet temperatures: both sides must be Dirichlet walls")
    tw = [float(v) for v in T_walls.detach().cpu().tolist()]
    if len(tw) != 2:
        raise ValueError("T_walls holds two values: (T_W, T_E)")
    tbc = list(p["T_bc"])
    tbc[0], tbc[1] = tw[0], tw[1]
    p["T_bc"] = tuple(tbc)
    lat = lbm.Lattice(p, precision, device=eps_field.device.index if eps_field.is_cuda else 0)
    e = eps_field.detach()
    if e.is_cuda and e.dtype == torch.float64:
        lat.set_fields(eps_field=e.contiguous())
    else:
        lat.set_fields(eps_field=e.cpu().numpy().astype(np.float64))
    return lat


class WallNusselt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_field, T_walls, problem, steps, precision, side, segment):
        lat = _lattice(eps_field, T_walls, problem, precision)
        try:
            lat.step(steps)
            loss, _ = lat.nusselt(side)
        finally:
            lat.close()
        ctx.save_for_backward(eps_field, T_walls)
        ctx.args = (problem, steps, precision, side, segment)
        return torch.tensor(loss, dtype=torch.float64, device=eps_field.device)

    @staticmethod
    def backward(ctx, grad):
        eps_field, T_walls = ctx.saved_tensors
        problem, steps, precision, side, segment = ctx.args
        need_eps, need_t = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_eps or need_t):
            return (None,) * 7
        lat = _lattice(eps_field, T_walls, problem, precision)
        try:
            _, g_eps, g_t = lat.adjoint(steps, side=side, segment=segment, porosity_gradient=need_eps)
        finally:
            lat.close()
        d_eps = d_t = None
        if need_eps:
            d_eps = grad.to(eps_field.device, torch.float64) * torch.from_numpy(g_eps).to(eps_field.device)
            d_eps = d_eps.to(eps_field.dtype)
        if need_t:
            d_t = grad.to(T_walls.device, torch.float64) * torch.tensor(g_t[:2], dtype=torch.float64,
                                                                        device=T_walls.device)
            d_t = d_t.to(T_walls.dtype)
        return d_eps, d_t, None, None, None, None, None


def wall_nusselt(eps_field: torch.Tensor, T_walls: torch.Tensor, problem: dict, steps: int,
                 precision: str = "f32", side: str = "W", segment: int = 0) -> torch.Tensor:
    return WallNusselt.apply(eps_field, T_walls, problem, steps, precision, side, segment)
