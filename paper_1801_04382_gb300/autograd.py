"""torch.autograd binding of the trajectory functional.

``KrotovTrajFunction.apply(eps, problem)`` returns J_T = 1 - F (Eq. functional_traj) for the
pulse ``eps`` [n_ctrl, nt] (float64 tensor); its backward is the library's gradient sweep
(co-state propagation along each trajectory's frozen jump record with exact propagator
derivatives, ``krotov_gradient``), i.e. dJ_T/deps with the record of this forward pass fixed.
Both directions run in the CUDA library; torch only carries the tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from .problem import Problem


class KrotovTrajFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps: torch.Tensor, problem: Problem):
        e = eps.detach().to("cpu", torch.float64).numpy()
        problem.set_pulses(e)
        F = problem.forward(keep_for_gradient=True)
        ctx.problem = problem
        ctx.eps_device = eps.device
        return torch.tensor(1.0 - F, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = ctx.problem.gradient()
        gt = torch.from_numpy(np.ascontiguousarray(g)).to(ctx.eps_device)
        return grad_out * gt, None


def trajectory_functional(eps: torch.Tensor, problem: Problem) -> torch.Tensor:
    """J_T(eps) with autograd support (see KrotovTrajFunction)."""
    return KrotovTrajFunction.apply(eps, problem)
