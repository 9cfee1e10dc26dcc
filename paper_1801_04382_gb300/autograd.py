"""torch.autograd binding of the trajectory functional.

``KrotovTrajFunction.apply(eps, problem)`` returns J_T = 1 - F (Eq. functional_traj) for the
pulse ``eps`` [n_ctrl, nt] (a CUDA float64 tensor); its backward is the library's gradient sweep
(co-state propagation along each trajectory's frozen jump record with exact propagator
derivatives, ``krotov_gradient``), i.e. dJ_T/deps with the record of this forward pass fixed.
Both directions run in the CUDA library on torch's current stream; the pulse, J_T and the
gradient stay in device memory (pointers cross the C ABI, nothing goes through the host).

The gradient belongs to the forward sweep of the same graph node: if the problem has run another
forward sweep since (a second evaluation, a line search, ``set_pulses``), backward raises instead
of returning the newer sweep's gradient.
"""
from __future__ import annotations

import torch

from .problem import Problem


class KrotovTrajFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps: torch.Tensor, problem: Problem):
        if not eps.is_cuda:
            raise ValueError("eps must be a CUDA tensor")
        stream = torch.cuda.current_stream(eps.device)
        e = eps.detach().to(torch.float64).contiguous()
        problem.set_pulses_device(e, stream=stream)
        problem.forward(keep_for_gradient=True, stream=stream, want_F=False)
        JT = problem.JT_device(stream=stream)
        ctx.problem = problem
        ctx.sweep = problem.sweeps()
        ctx.eps_dtype = eps.dtype
        return JT.to(eps.dtype)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        p = ctx.problem
        if p.sweeps() != ctx.sweep:
            raise RuntimeError("the problem ran another forward sweep after this J_T was evaluated; its "
                               "gradient belongs to the latest sweep -- evaluate J_T again before backward")
        g = p.gradient(stream=torch.cuda.current_stream(grad_out.device))
        return (grad_out * g).to(ctx.eps_dtype), None


def trajectory_functional(eps: torch.Tensor, problem: Problem) -> torch.Tensor:
    """J_T(eps) with autograd support (see KrotovTrajFunction)."""
    return KrotovTrajFunction.apply(eps, problem)
