"""Density-matrix Krotov optimisation (Sec. 2.2, Eqs. krotov_functional, krotovupdate,
krotov_boundary), FP64 -- the convergence reference of the trajectory formulations.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

    J_T = 1 - <<P_tgt|rho(T)>> = 1 - <tgt|rho(T)|tgt>                   (Eq. functional)
    P(T) = P_tgt = |tgt><tgt|                                            (Eq. krotov_boundary)
    Delta u_i(t) = S_i(t) / lambda_i  Im <<P^(0)(t)| dL/du_i |rho^(1)(t)>>  (Eq. krotovupdate)

with <<A|B>> = tr(A^dag B) and, as the paper states for the dissipator of Eq. lindblad,
dL/du_i rho = [H_i, rho].  rho^(1) runs forward under the updated controls (sequential in time),
P^(0) backward under the adjoint of the guess controls' dynamics: with E_j = exp(dt L_j) the
Liouville-space map of interval j (row-major vectorisation, ``lindblad.liouvillian``),
vec P(t_{j-1}) = E_j^dag vec P(t_j), so that <<P(t)|rho(t)>> is the same at every t under one
pulse.  Time discretisation as for the trajectory update: interval j uses P^(0)(t_{j-1}) and
rho^(1)(t_{j-1}) and the shape at its midpoint.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .lindblad import liouvillian


def _maps(model, eps: np.ndarray, dt: float) -> list:
    return [scipy.linalg.expm(dt * liouvillian(model.Heff(eps[:, j]), model.L).toarray())
            for j in range(eps.shape[1])]


def backward_P(model, eps: np.ndarray, T: float, P_T: np.ndarray) -> np.ndarray:
    """P(t_j), j = 0..nt, under the pulse eps [n_ctrl, nt]."""
    nt = eps.shape[1]
    E = _maps(model, eps, T / nt)
    d = P_T.shape[0]
    out = [None] * (nt + 1)
    v = np.asarray(P_T, dtype=np.complex128).ravel()
    out[nt] = v.reshape(d, d)
    for j in range(nt, 0, -1):
        v = E[j - 1].conj().T @ v
        out[j - 1] = v.reshape(d, d)
    return np.array(out)


def forward_update(model, eps: np.ndarray, T: float, rho0: np.ndarray, P: np.ndarray,
                   shape: np.ndarray, lam: np.ndarray):
    """Sequential update: returns (new eps, Delta eps, rho(T))."""
    n_ctrl, nt = eps.shape
    dt = T / nt
    new = np.array(eps, dtype=np.float64)
    deps = np.zeros_like(new)
    rho = np.asarray(rho0, dtype=np.complex128)
    d = rho.shape[0]
    for j in range(1, nt + 1):
        for i in range(n_ctrl):
            comm = model.Hc[i] @ rho - rho @ model.Hc[i]              # dL/du_i rho = [H_i, rho]
            deps[i, j - 1] = shape[i, j - 1] / lam[i] * np.imag(np.trace(P[j - 1].conj().T @ comm))
        new[:, j - 1] = eps[:, j - 1] + deps[:, j - 1]
        E = scipy.linalg.expm(dt * liouvillian(model.Heff(new[:, j - 1]), model.L).toarray())
        rho = (E @ rho.ravel()).reshape(d, d)
    return new, deps, rho


def functional(model, rho_T: np.ndarray) -> float:
    """J_T = 1 - <tgt|rho(T)|tgt>."""
    return 1.0 - float(np.real(np.vdot(model.psi_tgt, rho_T @ model.psi_tgt)))


def optimize_dm(model, eps0: np.ndarray, T: float, shape: np.ndarray, lam: np.ndarray, n_iter: int,
                rho0: np.ndarray = None):
    """n_iter density-matrix Krotov iterations; returns (J_T history incl. the guess, final eps)."""
    from .lindblad import propagate_rho
    rho0 = np.outer(model.psi0, model.psi0.conj()) if rho0 is None else rho0
    P_T = np.outer(model.psi_tgt, model.psi_tgt.conj())
    eps = np.array(eps0, dtype=np.float64)
    JT = [functional(model, propagate_rho(model, eps, T, rho0, dense=True))]
    for _ in range(n_iter):
        P = backward_P(model, eps, T, P_T)
        eps, _, rho_T = forward_update(model, eps, T, rho0, P, shape, lam)
        JT.append(functional(model, rho_T))
    return np.array(JT), eps
