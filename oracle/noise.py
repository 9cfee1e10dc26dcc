"""Noise measure of an optimised control field (Eq. noise, Sec. 4), FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

    nu_i = int_0^T |Omega_i(t) - Omega_i^smooth(t)| dt,

with Omega^smooth a five-point cubic Savitzky-Golay smoothing (the paper's choice of window and
polynomial order).  Written from the definition of the filter: at every sample j the cubic that
fits the five samples around j in the least-squares sense is evaluated at j; at the first and
last two samples, where no centred window exists, the cubic fitted to the first (last) five
samples is evaluated there.  The integral over the piecewise-constant control is the sum over
intervals times dt.
"""
from __future__ import annotations

import numpy as np


def savitzky_golay_cubic5(y: np.ndarray) -> np.ndarray:
    """Five-point cubic least-squares smoothing of a 1-D sequence (len >= 5)."""
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    if n < 5:
        raise ValueError("five-point smoothing needs at least five samples")
    out = np.empty(n)
    for j in range(n):
        start = min(max(j - 2, 0), n - 5)
        x = np.arange(start, start + 5, dtype=np.float64) - j      # window abscissae relative to j
        coef = np.polyfit(x, y[start:start + 5], 3)               # least-squares cubic
        out[j] = np.polyval(coef, 0.0)
    return out


def pulse_noise(eps: np.ndarray, dt: float) -> np.ndarray:
    """nu_i for every control row of eps [n_ctrl, nt] (Eq. noise)."""
    eps = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    return np.array([np.sum(np.abs(e - savitzky_golay_cubic5(e))) * dt for e in eps])


def fit_power_law(M: np.ndarray, nu: np.ndarray) -> float:
    """Exponent b of nu ~ M^b by least squares in log-log (Fig. 4 expects b = -1/2)."""
    b, _ = np.polyfit(np.log(np.asarray(M, dtype=np.float64)), np.log(np.asarray(nu, dtype=np.float64)), 1)
    return float(b)
