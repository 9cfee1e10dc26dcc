"""Exact gradient dJ_T/deps_ij of the trajectory functional with a frozen jump record, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper notes (Sec. 2.3) that a GRAPE-style gradient does not decompose into trajectories
because of the random jump times.  This build defines the differentiable object by freezing
the jump record R = {(step, s*, channel)} of a forward pass: then every trajectory is a fixed
product of step propagators and jump operators,
    psi_k(T) = U_{k,nt} ... U_{k,1} psi_0,   U_kj = P(tau_m) c_m L_m ... c_1 L_1 P(tau_0),
with P(tau) = expm(-i H_eff(eps_j) tau) and tau_q the free pieces between jumps.  The
functional of Eq. (functional_traj), J_T = 1 - (1/M) sum_k |<tgt|psi_k>|^2 / ||psi_k||^2,
is scale-invariant in psi_k so the c's drop out, and (Eq. gradient's "discrete exact
derivative", Sec. 2.2)
    dJ_T/deps_ij = -(1/M) sum_k 2 Re <chi~_k(t_j)| dU_kj/deps_i |psi_k(t_{j-1})>,
    chi~_k(T) = (tau_k |tgt> - |tau_k|^2 psihat_k) / ||psi_k(T)||,  chi~_k(t_{j-1}) = U_kj^dag chi~_k(t_j).
dP/deps_i is the top-right block of expm(-i tau [[H_eff, H_i], [0, H_eff]]) (block-triangular
augmented generator), applied to [0; psi].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mcwf import backward_pass
from .propagate import StepPropagator


def _records_by_step(records):
    out = {}
    for k, recs in enumerate(records):
        for rec in recs:
            out.setdefault((rec.step, k), []).append(rec)
    for key in out:
        out[key].sort(key=lambda r: r.s)
    return out


def frozen_forward(model, eps: np.ndarray, T: float, psi0: np.ndarray, records: list) -> np.ndarray:
    """States psi_k(t_j), j = 0..nt, replaying a fixed jump record.  Returns [nt+1, M, d]."""
    n_ctrl, nt = eps.shape
    M = len(records)
    d = model.d
    dt = T / nt
    by_step = _records_by_step(records)
    out = np.empty((nt + 1, M, d), dtype=np.complex128)
    out[0] = np.broadcast_to(psi0, (M, d))
    for j in range(1, nt + 1):
        prop = StepPropagator(model.Heff(eps[:, j - 1]))
        for k in range(M):
            psi = out[j - 1, k]
            t_lo = 0.0
            for rec in by_step.get((j, k), []):
                psi = prop.apply(psi, rec.s - t_lo)
                psi = rec.c * (model.L[rec.channel] @ psi)
                t_lo = rec.s
            out[j, k] = prop.apply(psi, dt - t_lo)
    return out


def jt_of_states(psi_T: np.ndarray, psi_tgt: np.ndarray) -> float:
    nrm2 = np.sum(np.abs(psi_T) ** 2, axis=1)
    ov = psi_T.conj() @ psi_tgt
    return float(1.0 - np.mean(np.abs(ov) ** 2 / nrm2))


def jt_frozen(model, eps, T, psi0, records) -> float:
    return jt_of_states(frozen_forward(model, eps, T, psi0, records)[-1], model.psi_tgt)


def gradient(model, eps: np.ndarray, T: float, psi0: np.ndarray, records: list):
    """dJ_T/deps [n_ctrl, nt] and J_T for the frozen record ``records``."""
    n_ctrl, nt = eps.shape
    M = len(records)
    d = model.d
    dt = T / nt
    psi_t = frozen_forward(model, eps, T, psi0, records)
    psi_T = psi_t[-1]
    nrm = np.sqrt(np.sum(np.abs(psi_T) ** 2, axis=1))
    psihat = psi_T / nrm[:, None]
    tau = (psihat.conj() @ model.psi_tgt).conj()
    chi_T = (tau[:, None] * model.psi_tgt[None, :] - (np.abs(tau) ** 2)[:, None] * psihat) / nrm[:, None]
    chi = backward_pass(model, eps, T, chi_T, records)
    by_step = _records_by_step(records)
    grad = np.zeros((n_ctrl, nt))
    for j in range(1, nt + 1):
        Heff = model.Heff(eps[:, j - 1])
        prop = StepPropagator(Heff)
        aug = []
        for i in range(n_ctrl):
            A = sp.bmat([[sp.csr_matrix(Heff), sp.csr_matrix(model.Hc[i])],
                         [None, sp.csr_matrix(Heff)]], format="csr")
            aug.append(StepPropagator(A if 2 * d > 162 else A.toarray(), dense_max=162))
        for k in range(M):
            recs = by_step.get((j, k), [])
            # pieces: P(tau_0), J_1, P(tau_1), ..., J_m, P(tau_m)
            taus, jumps = [], []
            t_lo = 0.0
            for rec in recs:
                taus.append(rec.s - t_lo)
                jumps.append(rec)
                t_lo = rec.s
            taus.append(dt - t_lo)
            for i in range(n_ctrl):
                # d(U psi) = sum_q [pieces after q] dP(tau_q) [pieces before q] psi
                val = 0.0
                for q in range(len(taus)):
                    v = psi_t[j - 1, k]
                    for p in range(q):
                        v = prop.apply(v, taus[p])
                        v = jumps[p].c * (model.L[jumps[p].channel] @ v)
                    z = np.concatenate([np.zeros(d, dtype=np.complex128), v])
                    dv = aug[i].apply(z, taus[q])[:d] if taus[q] > 0 else np.zeros(d, dtype=np.complex128)
                    for p in range(q, len(jumps)):
                        dv = jumps[p].c * (model.L[jumps[p].channel] @ dv)
                        dv = prop.apply(dv, taus[p + 1])
                    val += np.vdot(chi[j, k], dv)
                grad[i, j - 1] += -2.0 / M * float(np.real(val))
    return grad, jt_of_states(psi_T, model.psi_tgt)


def fd_gradient(model, eps, T, psi0, records, slots, h: float = 1e-4) -> np.ndarray:
    """Central finite differences of the frozen-record J_T at the given (i, j0) slots (0-based j0)."""
    out = []
    for (i, j0) in slots:
        ep = eps.copy(); ep[i, j0] += h
        em = eps.copy(); em[i, j0] -= h
        out.append((jt_frozen(model, ep, T, psi0, records) - jt_frozen(model, em, T, psi0, records)) / (2 * h))
    return np.array(out)
