"""Density-matrix reference for the trajectory average, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (lindblad) of the paper, written with the MCWF generator: for H_eff = H - (i/2) sum L^dag L,
    d rho / dt = -i (H_eff rho - rho H_eff^dag) + sum_l L_l rho L_l^dag,
which is -i[H, rho] + sum_l (L rho L^dag - 1/2 {L^dag L, rho}).  The trajectory expansion
Eq. (rho_traj_expansion) states that the average of |psihat_k><psihat_k| over M -> infinity
trajectories equals rho(t).

rho is row-major vectorised: vec(A X B) = (A (x) B^T) vec(X), so the Liouvillian is
    Lv = -i (H_eff (x) 1 - 1 (x) conj(H_eff)) + sum_l L_l (x) conj(L_l),
propagated over each piecewise-constant interval with scipy's expm_multiply (a library
routine) or, for tiny d, dense expm.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def liouvillian(Heff: np.ndarray, Ls: list) -> sp.csr_matrix:
    d = Heff.shape[0]
    one = sp.identity(d, format="csr", dtype=np.complex128)
    Hs = sp.csr_matrix(Heff)
    out = -1j * (sp.kron(Hs, one) - sp.kron(one, Hs.conj()))
    for l_op in Ls:
        Ls_ = sp.csr_matrix(l_op)
        out = out + sp.kron(Ls_, Ls_.conj())
    return sp.csr_matrix(out)


def propagate_rho(model, eps: np.ndarray, T: float, rho0: np.ndarray, dense: bool = False,
                  keep: bool = False):
    """rho(T) (or all rho(t_j) if keep) under piecewise-constant eps [n_ctrl, nt]."""
    n_ctrl, nt = eps.shape
    dt = T / nt
    v = np.asarray(rho0, dtype=np.complex128).ravel()
    traj = [v.reshape(rho0.shape).copy()] if keep else None
    for j in range(nt):
        Lv = liouvillian(model.Heff(eps[:, j]), model.L)
        if dense:
            v = scipy.linalg.expm(dt * Lv.toarray()) @ v
        else:
            v = spla.expm_multiply(dt * Lv, v)
        if keep:
            traj.append(v.reshape(rho0.shape).copy())
    return np.array(traj) if keep else v.reshape(rho0.shape)
