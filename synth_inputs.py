"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds *inputs only*: workload sizes, seeded uniform random numbers,
guess pulses, shape functions and random initial states.  It contains none of
the method's arithmetic (no Hamiltonian, no propagation, no update), so that
the FP64 oracle (``oracle/``) and the CUDA path can both be fed from it without
sharing any computation.

Workloads follow the five cascaded atom-cavity configurations of the build
plan: N nodes, each a three-level atom {g, e, r} in a cavity truncated at
``n_cav`` photons (local dimension 3*(n_cav+1), d = n_loc**N), energies in
units of g, time in units of hbar/g, Delta = 100 g and kappa = g (Sec. 3.2 of
the paper), T = 50, a sin^2 guess pulse of amplitude 1 on every node's control
and the same sin^2 shape function S(t), lambda = 10.

Random numbers (Sec. 2.1, the MCWF algorithm): each forward pass ``p`` and each
trajectory ``k`` owns a row ``U[p, k, :]`` of ``1 + 2*max_jumps`` uniforms in
[0, 1).  Column 0 is the first norm threshold r; after the m-th jump (m = 1,
2, ...) column 2m-1 chooses the Lindblad channel and column 2m is the next r.
Both implementations read the same array; no device RNG is on the parity path.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic optimisation problem (model + run parameters)."""
    name: str
    n_nodes: int
    n_cav: int                  # cavity truncation: photon numbers 0..n_cav
    T: float
    nt: int
    M: int                      # number of trajectories
    seed: int
    n_iter: int = 1             # Krotov iterations the workload asks for
    delta: float = 100.0        # atom-laser detuning Delta (units of g)
    g: float = 1.0              # atom-cavity coupling
    kappa: float = 1.0          # cavity decay rate
    lam: float = 10.0           # Krotov step weight lambda_i (all controls)
    guess_amp: float = 1.0      # guess pulse amplitude (units of g)
    precision: str = "fp64"     # "fp64" or "fp32"
    ckpt_interval: int = 0      # 0: store the co-state at every step
    max_jumps: int = 0          # 0: use the excitation bound n_nodes*(1+n_cav)

    @property
    def n_loc(self) -> int:
        return 3 * (self.n_cav + 1)

    @property
    def d(self) -> int:
        return self.n_loc ** self.n_nodes

    @property
    def dt(self) -> float:
        return self.T / self.nt

    @property
    def jumps_cap(self) -> int:
        return self.max_jumps if self.max_jumps > 0 else self.n_nodes * (1 + self.n_cav)

    @property
    def draws_per_traj(self) -> int:
        return 1 + 2 * self.jumps_cap

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# The five workloads (sizes as specified for this method's benchmark suite).
CONFIGS = {
    "cfg1_d36": Workload("cfg1_d36", n_nodes=2, n_cav=1, T=50.0, nt=500, M=32, seed=0,
                         n_iter=1, precision="fp64"),
    "cfg2_d81": Workload("cfg2_d81", n_nodes=2, n_cav=2, T=50.0, nt=1000, M=128, seed=1,
                         n_iter=50, precision="fp64"),
    "cfg3_d729": Workload("cfg3_d729", n_nodes=3, n_cav=2, T=50.0, nt=2000, M=1024, seed=2,
                          n_iter=1, precision="fp32"),
    "cfg5_d6561": Workload("cfg5_d6561", n_nodes=4, n_cav=2, T=50.0, nt=5000, M=1024, seed=4,
                           n_iter=20, precision="fp32", ckpt_interval=100),
}


def uniforms(seed: int, n_passes: int, M: int, draws_per_traj: int) -> np.ndarray:
    """FP64 uniforms in [0, 1), shape [n_passes, M, draws_per_traj]."""
    return np.random.default_rng(seed).random((n_passes, M, draws_per_traj))


def midpoints(nt: int, T: float) -> np.ndarray:
    """Midpoints t_{j-1/2} of the nt piecewise-constant control intervals."""
    return (np.arange(nt, dtype=np.float64) + 0.5) * (T / nt)


def sin2_envelope(nt: int, T: float) -> np.ndarray:
    """sin^2(pi t / T) sampled at the interval midpoints."""
    return np.sin(np.pi * midpoints(nt, T) / T) ** 2


def guess_pulses(n_ctrl: int, nt: int, T: float, amp: float) -> np.ndarray:
    """Guess controls eps_i^(0)(t_{j-1/2}) = amp * sin^2(pi t / T), shape [n_ctrl, nt]."""
    return np.tile(amp * sin2_envelope(nt, T), (n_ctrl, 1))


def shape_functions(n_ctrl: int, nt: int, T: float) -> np.ndarray:
    """Update shape S_i(t_{j-1/2}) = sin^2(pi t / T) in [0, 1], shape [n_ctrl, nt]."""
    return np.tile(sin2_envelope(nt, T), (n_ctrl, 1))


def random_pulses(seed: int, n_ctrl: int, nt: int, scale: float) -> np.ndarray:
    """Smooth-ish random controls (sum of a few sines), shape [n_ctrl, nt]."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nt) + 0.5) / nt
    out = np.zeros((n_ctrl, nt))
    for i in range(n_ctrl):
        for m in range(1, 4):
            out[i] += rng.normal() * np.sin(math.pi * m * x + rng.uniform(0, 2 * math.pi))
    return scale * out


def random_states(seed: int, M: int, d: int) -> np.ndarray:
    """M normalised complex states with iid Gaussian amplitudes, shape [M, d]."""
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(M, d)) + 1j * rng.normal(size=(M, d))
    return z / np.linalg.norm(z, axis=1, keepdims=True)


def batch_mix(seed: int = 3, n: int = 64, hbm_budget: float = 150e9, n_iter: int = 1) -> list:
    """A batch of n independent problems of mixed size: N in {2, 3, 4} nodes with cavity cutoff 2
    (d = 81, 729, 6561), M = 2**U{7..11} trajectories, nt in {1000, 2000} (T = 50), kappa ~ U[0.5, 2],
    FP32-mixed.  Co-states are kept at every step where the batch fits ``hbm_budget`` bytes;
    otherwise the problems holding the most co-state memory are switched, largest first, to
    checkpoints every round(sqrt(nt)) steps, which minimises checkpoints + segment buffer."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.integers(2, 5))
        M = 2 ** int(rng.integers(7, 12))
        nt = int(rng.choice([1000, 2000]))
        kappa = float(rng.uniform(0.5, 2.0))
        out.append(Workload(f"mix{i:02d}_N{N}_M{M}_nt{nt}", n_nodes=N, n_cav=2, T=50.0, nt=nt, M=M,
                            seed=seed * 1000 + i, n_iter=n_iter, kappa=kappa, precision="fp32"))

    def held(w):
        return costate_bytes(w) + 4 * w.M * w.d * 8     # co-states + initial/running states

    total = sum(held(w) for w in out)
    for i in sorted(range(n), key=lambda i: -held(out[i])):
        if total <= hbm_budget:
            break
        before = held(out[i])
        out[i] = out[i].with_(ckpt_interval=int(round(math.sqrt(out[i].nt))))
        total += held(out[i]) - before
    return out


def costate_bytes(w: Workload) -> int:
    """Device bytes of the co-state storage of workload w in its precision: every step, or
    checkpoints every ckpt_interval steps plus the segment buffer."""
    state = w.M * w.d * (8 if w.precision == "fp32" else 16)
    if w.ckpt_interval == 0:
        return (w.nt + 1) * state
    K = w.ckpt_interval
    return (w.nt // K + 1 + (1 if w.nt % K else 0) + K + 1) * state
