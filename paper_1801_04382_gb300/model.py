"""Structured description of a cascaded atom-cavity network (paper Sec. 3.1).

Produces the node-local factors, pair list and Lindblad coefficients that the C ABI takes
(``kt_model_desc``); the full d x d operators are never formed.

Node = three-level atom {g, e, r} in a cavity truncated at ``n_cav`` photons; local index
atom * (n_cav + 1) + n (g = 0, e = 1, r = 2); node 0 is the most significant factor.
Node Hamiltonian (explicit three-level model whose adiabatic elimination of r yields the
paper's effective node Hamiltonian H_0 + H_d):
    h = -Delta |r><r| - (g^2 / Delta) a^dag a + g (|r><g| a + |g><r| a^dag),
control eps_c on node c (the Raman drive Omega_c):  dH/deps_c = (i/2)(|r><e| - |e><r|).
Cascade (Eq. ham_interaction): for i < j,  i kappa a_i^dag a_j - i kappa a_j^dag a_i.
One collective Lindblad operator L = sqrt(2 kappa) sum_i a_i.
Initial state |e g .. g>|0 .. 0>, target the W state (1/sqrt N) sum_i |g..e_i..g>|0..0>.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

ATOM_G, ATOM_E, ATOM_R = 0, 1, 2


@dataclass
class NetworkFactors:
    n_nodes: int
    n_loc: int
    h0_local: np.ndarray          # [N, n_loc, n_loc] complex
    hc_local: np.ndarray          # [n_ctrl, n_loc, n_loc] complex
    ctrl_node: np.ndarray         # [n_ctrl] int
    a_local: np.ndarray           # [n_loc, n_loc] complex
    pair_dst: np.ndarray          # [P] int
    pair_src: np.ndarray          # [P] int
    pair_coef: np.ndarray         # [P] complex
    lind_coef: np.ndarray         # [n_lind, N] complex
    psi0: np.ndarray              # [d] complex
    psi_tgt: np.ndarray           # [d] complex

    @property
    def d(self) -> int:
        return self.n_loc ** self.n_nodes

    @property
    def n_ctrl(self) -> int:
        return len(self.ctrl_node)


def _loc(n_cav: int, atom: int, n: int) -> int:
    return atom * (n_cav + 1) + n


def _full_index(n_loc: int, digits) -> int:
    x = 0
    for dgt in digits:
        x = x * n_loc + dgt
    return x


def cascaded_chain(n_nodes: int, n_cav: int, delta: float = 100.0, g: complex = 1.0,
                   kappa: float = 1.0, lindblad: str = "collective") -> NetworkFactors:
    """``lindblad``: "collective" -- the network's single output L = sqrt(2 kappa) sum_i a_i;
    "local" -- one operator per node, L_i = sqrt(2 kappa) a_i (every cavity's output detected on its
    own, n_lind = n_nodes)."""
    if lindblad not in ("collective", "local"):
        raise ValueError("lindblad must be 'collective' or 'local'")
    nl = 3 * (n_cav + 1)
    a = np.zeros((nl, nl), dtype=np.complex128)
    h = np.zeros((nl, nl), dtype=np.complex128)
    hc = np.zeros((nl, nl), dtype=np.complex128)
    for atom in (ATOM_G, ATOM_E, ATOM_R):
        for n in range(n_cav + 1):
            x = _loc(n_cav, atom, n)
            if n >= 1:
                a[_loc(n_cav, atom, n - 1), x] = math.sqrt(n)          # a |n> = sqrt(n) |n-1>
            h[x, x] += -(abs(g) ** 2 / delta) * n
            if atom == ATOM_R:
                h[x, x] += -delta
    for n in range(1, n_cav + 1):
        # g |r, n-1><g, n| sqrt(n)  (|r><g| a)  and its Hermitian conjugate (g may carry a phase)
        r_, g_ = _loc(n_cav, ATOM_R, n - 1), _loc(n_cav, ATOM_G, n)
        h[r_, g_] += g * math.sqrt(n)
        h[g_, r_] += np.conj(g) * math.sqrt(n)
    for n in range(n_cav + 1):
        r_, e_ = _loc(n_cav, ATOM_R, n), _loc(n_cav, ATOM_E, n)
        hc[r_, e_] += 0.5j
        hc[e_, r_] += -0.5j
    pd, ps, pc = [], [], []
    for i in range(n_nodes):
        for j in range(i + 1, n_nodes):
            pd += [i, j]
            ps += [j, i]
            pc += [1j * kappa, -1j * kappa]
    d = nl ** n_nodes
    psi0 = np.zeros(d, dtype=np.complex128)
    psi0[_full_index(nl, [_loc(n_cav, ATOM_E, 0)] + [_loc(n_cav, ATOM_G, 0)] * (n_nodes - 1))] = 1.0
    tgt = np.zeros(d, dtype=np.complex128)
    for i in range(n_nodes):
        digits = [_loc(n_cav, ATOM_G, 0)] * n_nodes
        digits[i] = _loc(n_cav, ATOM_E, 0)
        tgt[_full_index(nl, digits)] = 1.0 / math.sqrt(n_nodes)
    return NetworkFactors(
        n_nodes=n_nodes, n_loc=nl,
        h0_local=np.repeat(h[None], n_nodes, axis=0),
        hc_local=np.repeat(hc[None], n_nodes, axis=0),
        ctrl_node=np.arange(n_nodes, dtype=np.int32),
        a_local=a,
        pair_dst=np.array(pd, dtype=np.int32), pair_src=np.array(ps, dtype=np.int32),
        pair_coef=np.array(pc, dtype=np.complex128),
        lind_coef=(np.full((1, n_nodes), math.sqrt(2.0 * kappa), dtype=np.complex128) if lindblad == "collective"
                   else math.sqrt(2.0 * kappa) * np.eye(n_nodes, dtype=np.complex128)),
        psi0=psi0, psi_tgt=tgt,
    )
