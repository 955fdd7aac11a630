"""PyTorch autograd interface to the discrete adjoint (``lbm_adjoint``).

``wall_nusselt(eps_field, T_walls, problem, steps)`` returns the mean
Nusselt number on the hot (W) wall after ``steps`` steps as a differentiable
scalar of the porosity field and of the two Dirichlet wall temperatures
(T_W, T_E).  The forward pass runs the whole checkpointed forward and
adjoint in one ``lbm_adjoint`` call (checkpoints every ceil(sqrt(steps))
steps, states recomputed from them) and keeps the gradients; ``backward``
scales them by the incoming gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class WallNusselt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_field, T_walls, problem, steps, precision, side, segment):
        p = dict(problem)
        tw = [float(v) for v in T_walls.detach().cpu().tolist()]
        tbc = list(p["T_bc"])
        tbc[0], tbc[1] = tw[0], tw[1]
        p["T_bc"] = tuple(tbc)
        lat = lbm.Lattice(p, precision, device=eps_field.device.index if eps_field.is_cuda else 0)
        try:
            lat.set_fields(eps_field=eps_field.detach().cpu().numpy().astype(np.float64))
            loss, g_eps, g_t = lat.adjoint(steps, side=side, segment=segment)
        finally:
            lat.close()
        ctx.save_for_backward(torch.from_numpy(g_eps).to(eps_field), torch.tensor(g_t[:2]).to(T_walls))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad):
        g_eps, g_t = ctx.saved_tensors
        g = grad.to(g_eps.dtype)
        return g * g_eps, g.to(g_t.dtype) * g_t, None, None, None, None, None


def wall_nusselt(eps_field: torch.Tensor, T_walls: torch.Tensor, problem: dict, steps: int,
                 precision: str = "f32", side: str = "W", segment: int = 0) -> torch.Tensor:
    return WallNusselt.apply(eps_field, T_walls, problem, steps, precision, side, segment)
