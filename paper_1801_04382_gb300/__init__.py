"""Trajectory-parallel Krotov optimisation on GB300 (Goerz & Jacobs, arXiv:1801.04382).

The hot path (batched MCWF forward propagation with norm-threshold jumps, backward co-state
propagation, per-step cross-trajectory pulse update) runs in hand-written CUDA for sm_103a
behind the C ABI of ``include/krotov_traj.h``; this package holds the build script, the
ctypes binding (``Problem``) and the structured model builder.
"""
from .model import NetworkFactors, cascaded_chain  # noqa: F401
from .problem import (Batch, DensityProblem, Problem, ShardGroup, bessel_j, nccl_unique_id,  # noqa: F401
                      shard_ranges)
from . import build  # noqa: F401  (module: build.build() compiles the CUDA library)
from ._capi import KrotovError  # noqa: F401


def __getattr__(name):
    # torch is only needed for the autograd binding
    if name in ("KrotovTrajFunction", "trajectory_functional"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
