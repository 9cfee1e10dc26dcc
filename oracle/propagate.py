"""Exact FP64 step propagators for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The controls are piecewise constant on the time grid (paper Sec. 2.2, "The control fields
are approximated as constant within the time interval"), so within one interval the
trajectory evolves under the fixed non-Hermitian generator H_eff(eps_j) and the exact
propagator over a duration tau is expm(-i H_eff tau) (Sec. 2.1, step 3 of the MCWF
algorithm, with hbar = 1).

* ``expm_propagator``: dense matrix exponential (scipy.linalg.expm), the plain definition.
  Used for d <= 81.
* ``ChebyshevPropagator``: FP64 Chebyshev expansion of exp(-i A tau) on a sparse matrix,
  for d > 81 where dense expm per step is too slow.  It is pinned against
  ``expm_propagator`` on d <= 81 in the tests.  Coefficients use scipy.special.jv.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.special


def expm_propagator(A: np.ndarray, tau: float) -> np.ndarray:
    """Dense expm(-i A tau)."""
    return scipy.linalg.expm(-1j * tau * np.asarray(A))


def gershgorin_bounds(A) -> tuple:
    """Bounds on the spectrum of a (possibly non-Hermitian) matrix A.

    Returns (e_min, e_max, damp): the real parts of all eigenvalues lie in [e_min, e_max]
    and their imaginary parts in [-damp, damp]; from Gershgorin discs of the Hermitian part
    (A + A^dag)/2 and the anti-Hermitian part (A - A^dag)/(2i).  The field of values of A is
    contained in that rectangle, hence so is the spectrum.
    """
    A = sp.csr_matrix(A)
    Ah = (A + A.getH()) * 0.5
    Aa = (A - A.getH()) * (-0.5j)
    def disc(B):
        B = sp.csr_matrix(B)
        diag = B.diagonal().real
        absrow = np.asarray(abs(B).sum(axis=1)).ravel() - np.abs(B.diagonal())
        return float(np.min(diag - absrow)), float(np.max(diag + absrow))
    lo, hi = disc(Ah)
    alo, ahi = disc(Aa)
    return lo, hi, max(abs(alo), abs(ahi))


class ChebyshevPropagator:
    """exp(-i A tau) v for a sparse A by a Chebyshev series (FP64).

    With A = c + r * Ahat, the spectrum of Ahat lies in an ellipse around [-1, 1] and
        exp(-i A tau) = exp(-i c tau) sum_k (2 - delta_k0) (-i)^k J_k(r tau) T_k(Ahat),
    the Chebyshev polynomials T_k obeying T_{k+1} = 2 Ahat T_k - T_{k-1}.  Terms are added
    until the coefficient, amplified by the growth rate of T_k on the ellipse that holds
    the (damped) spectrum, is below 1e-18.
    """

    def __init__(self, A, margin: float = 1.01):
        self.A = sp.csr_matrix(A)
        lo, hi, damp = gershgorin_bounds(self.A)
        self.c = 0.5 * (lo + hi)
        self.r = 0.5 * (hi - lo) * margin + 1e-12
        b = damp / self.r
        # Bernstein ellipse parameter rho of an ellipse (foci +-1) holding the
        # rectangle [-1, 1] x [-b, b] (checked at the corner 1 + i b).
        z = complex(1.0, b)
        w = z + np.sqrt(z - 1) * np.sqrt(z + 1)
        self.rho = max(abs(w), 1.0)
        d = self.A.shape[0]
        self.Ahat = (self.A - self.c * sp.identity(d, format="csr")) / self.r

    def coefficients(self, tau: float) -> np.ndarray:
        alpha = self.r * tau
        coefs = []
        k = 0
        while True:
            jk = scipy.special.jv(k, alpha)
            coefs.append((2.0 if k else 1.0) * (-1j) ** k * jk)
            if k > alpha and abs(jk) * self.rho ** k < 1e-18 and k >= 4:
                break
            k += 1
            if k > 10000:
                raise RuntimeError("Chebyshev series did not converge")
        return np.array(coefs) * np.exp(-1j * self.c * tau)

    def apply(self, v: np.ndarray, tau: float) -> np.ndarray:
        """exp(-i A tau) v for v of shape [d] or [d, m]."""
        a = self.coefficients(tau)
        t_prev = v
        out = a[0] * t_prev
        if len(a) == 1:
            return out
        t_cur = self.Ahat @ v
        out = out + a[1] * t_cur
        for k in range(2, len(a)):
            t_next = 2.0 * (self.Ahat @ t_cur) - t_prev
            out = out + a[k] * t_next
            t_prev, t_cur = t_cur, t_next
        return out


class StepPropagator:
    """exp(-i A tau) applied to vectors: dense expm for small d, Chebyshev otherwise."""

    def __init__(self, A, dense_max: int = 81):
        self.d = A.shape[0]
        self.dense = self.d <= dense_max
        if self.dense:
            self.A = np.asarray(A.toarray() if sp.issparse(A) else A)
            self._cache = {}
        else:
            self.cheb = ChebyshevPropagator(A)

    def matrix(self, tau: float) -> np.ndarray:
        if not self.dense:
            raise ValueError("dense propagator matrix requested for a large problem")
        key = float(tau)
        m = self._cache.get(key)
        if m is None:
            m = expm_propagator(self.A, tau)
            if len(self._cache) < 8:
                self._cache[key] = m
        return m

    def apply(self, v: np.ndarray, tau: float) -> np.ndarray:
        if tau == 0.0:
            return v.copy()
        if self.dense:
            return self.matrix(tau) @ v
        return self.cheb.apply(v, tau)

    def apply_adjoint(self, v: np.ndarray, tau: float) -> np.ndarray:
        """expm(-i A tau)^dag v."""
        if tau == 0.0:
            return v.copy()
        if self.dense:
            return self.matrix(tau).conj().T @ v
        # expm(-i A tau)^dag = expm(+i A^dag tau) = expm(-i (-A^dag) tau)
        if not hasattr(self, "_adj"):
            self._adj = ChebyshevPropagator(-self.cheb.A.getH())
        return self._adj.apply(v, tau)
