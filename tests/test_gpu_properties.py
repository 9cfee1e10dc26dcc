"""Properties of the GPU path that hold at any size, checked beyond the oracle's parity cases.

- Trajectory average -> master equation (the MCWF unravelling, Sec. 2.1): with 16384 trajectories
  and jumps, F = mean_k |tau_k|^2 equals <tgt|rho(T)|tgt> of the oracle's Lindblad propagation
  within 3 sigma / sqrt(M), and the fraction of trajectories that jumped equals 1 - ||psi_nojump(T)||^2
  within the binomial 3 sigma.
- Monotonic convergence (Sec. 2.2): in the deterministic case (kappa = 0) every Krotov iteration
  lowers J_T.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import synth_inputs as si
from oracle import lindblad as ol
from oracle import model as om
from paper_1801_04382_gb300 import Problem, cascaded_chain

pytestmark = pytest.mark.gpu


def test_trajectory_average_converges_to_lindblad():
    T, nt, M = 20.0, 200, 16384
    m = om.build_model(2, 1)
    eps = si.guess_pulses(2, nt, T, 40.0)
    with Problem(cascaded_chain(2, 1), T, nt, M, eps, si.shape_functions(2, nt, T), np.full(2, 10.0),
                 si.uniforms(21, 1, M, 5)) as p:
        F = p.forward(False)
        _, tau = p.fidelity()
        jumped = np.mean([len(r) > 0 for r in p.records()])
    rho = ol.propagate_rho(m, eps, T, np.outer(m.psi0, m.psi0.conj()))
    f_rho = float(np.vdot(m.psi_tgt, rho @ m.psi_tgt).real)
    sigma = np.std(np.abs(tau) ** 2)
    assert abs(F - f_rho) <= 3 * sigma / math.sqrt(M)
    psi = m.psi0.copy()
    for j in range(nt):
        psi = scipy.linalg.expm(-1j * m.Heff(eps[:, j]) * (T / nt)) @ psi
    p_jump = 1.0 - float(np.vdot(psi, psi).real)
    assert 0.05 < p_jump < 0.95
    assert abs(jumped - p_jump) <= 3 * math.sqrt(p_jump * (1 - p_jump) / M)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_krotov_monotone_at_kappa_zero(precision):
    nt, T = 200, 20.0
    eps = si.guess_pulses(2, nt, T, 30.0)
    with Problem(cascaded_chain(2, 2, kappa=0.0), T, nt, 1, eps, si.shape_functions(2, nt, T), np.full(2, 0.2),
                 si.uniforms(0, 9, 1, 13), precision=precision) as p:
        JT0 = 1.0 - p.forward(False)
        JT, _ = p.update(8)
    JT = np.concatenate([[JT0], JT])
    assert np.all(np.diff(JT) < 0.0)
    assert JT[-1] < JT[0] - 5e-4
