"""Dense FP64 operators of the cascaded atom-cavity network, by explicit Kronecker products.

TEST INFRASTRUCTURE ONLY: the oracle is imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of the benchmark, never by the product path.

Physics (paper Sec. 3.1, "Network Model", and the readings listed with this build):

* One node = three-level atom {g, e, r} in a cavity truncated at ``n_cav`` photons.
  Local basis index = atom * (n_cav + 1) + n with atom g=0, e=1, r=2 and n the photon
  number.  In the full space node 0 is the most significant factor.
* Node Hamiltonian (explicit three-level form whose adiabatic elimination of r gives the
  paper's effective H_0^(i) + H_d^(i)):
      h^(i) = -Delta Pi_r - (g^2/Delta) a^dag a + g (sigma_rg a + sigma_gr a^dag)
              + (i eps_i / 2)(sigma_re - sigma_er),
  the cavity driving g<->r, the laser eps_i = Omega_i driving r<->e.
* Cascade interaction between nodes i < j (Eq. ham_interaction):
      H^(i,j) = i kappa a_i^dag a_j - i kappa a_j^dag a_i.
* One collective Lindblad operator L = sqrt(2 kappa) sum_i a_i (Sec. 3.1).
* MCWF effective Hamiltonian (Sec. 2.1): H_eff = H - (i/2) sum_l L_l^dag L_l
  (the printed "+ sum L^dag L" is read as the standard -(i/2) L^dag L, since only that
  form makes the norm decay and allows jumps).
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import reduce

import numpy as np
import scipy.sparse as sp

G, E, R = 0, 1, 2  # atom levels
SPARSE_ABOVE = 729  # full-space dimension above which operators are held as scipy.sparse CSR


def atom_op(row: int, col: int) -> np.ndarray:
    """|row><col| on the three-level atom."""
    m = np.zeros((3, 3), dtype=np.complex128)
    m[row, col] = 1.0
    return m


def cavity_lowering(n_cav: int) -> np.ndarray:
    """Truncated annihilation operator a with a|n> = sqrt(n)|n-1>."""
    a = np.zeros((n_cav + 1, n_cav + 1), dtype=np.complex128)
    for n in range(1, n_cav + 1):
        a[n - 1, n] = np.sqrt(n)
    return a


def local_operators(n_cav: int) -> dict:
    """Single-node operators on atom (x) cavity, atom the more significant factor."""
    ia = np.eye(3, dtype=np.complex128)
    ic = np.eye(n_cav + 1, dtype=np.complex128)
    a = np.kron(ia, cavity_lowering(n_cav))
    return {
        "a": a,
        "n": a.conj().T @ a,
        "Pi_r": np.kron(atom_op(R, R), ic),
        "sigma_rg": np.kron(atom_op(R, G), ic),
        "sigma_re": np.kron(atom_op(R, E), ic),
        "id": np.kron(ia, ic),
    }


def embed(op, node: int, n_nodes: int, sparse: bool = False):
    """op acting on node ``node`` of ``n_nodes`` identical nodes (node 0 most significant)."""
    if sparse:
        ident = sp.identity(op.shape[0], dtype=np.complex128, format="csr")
        factors = [sp.csr_matrix(op) if i == node else ident for i in range(n_nodes)]
        return reduce(lambda x, y: sp.kron(x, y, format="csr"), factors)
    ident = np.eye(op.shape[0], dtype=np.complex128)
    factors = [op if i == node else ident for i in range(n_nodes)]
    return reduce(np.kron, factors)


@dataclass
class DenseModel:
    """All dense operators of one network instance."""
    n_nodes: int
    n_cav: int
    H0: np.ndarray          # drift Hamiltonian (Hermitian), incl. cascade terms
    Hc: list                # control Hamiltonians dH/deps_i (Hermitian), one per node
    L: list                 # Lindblad operators
    psi0: np.ndarray
    psi_tgt: np.ndarray

    @property
    def d(self) -> int:
        return self.H0.shape[0]

    def H(self, eps) -> np.ndarray:
        """Hermitian Hamiltonian H(eps) = H0 + sum_i eps_i Hc_i."""
        out = self.H0.copy()
        for e, hc in zip(eps, self.Hc):
            out = out + e * hc
        return out

    def LdagL(self):
        out = 0 * self.H0
        for l_op in self.L:
            out = out + l_op.conj().T @ l_op
        return out

    def Heff(self, eps) -> np.ndarray:
        """Non-Hermitian MCWF generator H_eff = H(eps) - (i/2) sum_l L_l^dag L_l."""
        return self.H(eps) - 0.5j * self.LdagL()


def basis_index(n_cav: int, atoms, photons) -> int:
    """Full-space index of the product state |atoms[0], photons[0]> (x) ... ."""
    n_loc = 3 * (n_cav + 1)
    idx = 0
    for a, n in zip(atoms, photons):
        idx = idx * n_loc + a * (n_cav + 1) + n
    return idx


def build_model(n_nodes: int, n_cav: int, delta: float = 100.0, g: complex = 1.0,
                kappa: float = 1.0, lindblad: str = "collective") -> DenseModel:
    """Cascaded chain of ``n_nodes`` atom-cavity nodes (paper Sec. 3.1).  A complex g = |g| e^(i phi)
    couples g sigma_rg a + conj(g) sigma_gr a^dag (a phase the paper's real g = 1 does not have,
    used to exercise complex couplings).

    ``lindblad``: "collective" -- the paper's single operator L = sqrt(2 kappa) sum_i a_i;
    "local" -- one operator per node, L_i = sqrt(2 kappa) a_i (the field leaving each cavity
    detected separately; not the paper's network, used to exercise the channel choice of Sec. 2.1
    with several Lindblad operators)."""
    loc = local_operators(n_cav)
    d = (3 * (n_cav + 1)) ** n_nodes
    sparse = d > SPARSE_ABOVE      # same operators, stored sparse so that d = 6561 fits in memory
    H0 = sp.csr_matrix((d, d), dtype=np.complex128) if sparse else np.zeros((d, d), dtype=np.complex128)
    a_full = [embed(loc["a"], i, n_nodes, sparse) for i in range(n_nodes)]
    h0_node = (-delta * loc["Pi_r"] - (abs(g) ** 2 / delta) * loc["n"]
               + g * (loc["sigma_rg"] @ loc["a"]) + np.conj(g) * (loc["sigma_rg"] @ loc["a"]).conj().T)
    for i in range(n_nodes):
        H0 = H0 + embed(h0_node, i, n_nodes, sparse)
    for i in range(n_nodes):
        for j in range(i + 1, n_nodes):
            H0 = H0 + 1j * kappa * (a_full[i].conj().T @ a_full[j])
            H0 = H0 + (-1j * kappa) * (a_full[j].conj().T @ a_full[i])
    hc_node = 0.5j * (loc["sigma_re"] - loc["sigma_re"].conj().T)
    Hc = [embed(hc_node, i, n_nodes, sparse) for i in range(n_nodes)]
    if lindblad == "collective":
        L = [np.sqrt(2.0 * kappa) * reduce(lambda x, y: x + y, a_full)]
    elif lindblad == "local":
        L = [np.sqrt(2.0 * kappa) * a_i for a_i in a_full]
    else:
        raise ValueError("lindblad must be 'collective' or 'local'")
    psi0 = np.zeros(d, dtype=np.complex128)
    psi0[basis_index(n_cav, [E] + [G] * (n_nodes - 1), [0] * n_nodes)] = 1.0
    tgt = np.zeros(d, dtype=np.complex128)
    for i in range(n_nodes):
        atoms = [G] * n_nodes
        atoms[i] = E
        tgt[basis_index(n_cav, atoms, [0] * n_nodes)] = 1.0
    tgt /= np.sqrt(n_nodes)
    return DenseModel(n_nodes, n_cav, H0, Hc, L, psi0, tgt)


def excitation_number(n_nodes: int, n_cav: int) -> np.ndarray:
    """Diagonal of N_exc = sum_i (Pi_e + Pi_r + a^dag a)_i over the full basis."""
    loc = local_operators(n_cav)
    ne = np.diag(np.kron(atom_op(E, E) + atom_op(R, R), np.eye(n_cav + 1))).real + np.diag(loc["n"]).real
    out = np.zeros((3 * (n_cav + 1)) ** n_nodes)
    for i in range(n_nodes):
        out += np.diag(embed(np.diag(ne).astype(np.complex128), i, n_nodes)).real
    return np.rint(out)
