"""Pulse noise (Eq. noise) computed on the device against the oracle's definition, on the pulse
of a short optimisation with jumps.  Both sides read the same (device) pulse, so the comparison
is of the smoothing and the integral alone.  nu sums |eps - smooth| over differences far smaller
than eps itself, so the bound is absolute: each smoothed sample is a five-term sum with weights of
total magnitude below 2.5, rounded to within a few ulp of max |eps| on either side; summed over
the nt intervals of length dt that is at most 16 eps_64 max|eps| T."""
import numpy as np
import pytest

import synth_inputs as si
from oracle import noise
from paper_1801_04382_gb300 import Problem, cascaded_chain

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pulse_noise_matches_oracle(precision):
    N, nc, T, nt, M = 2, 1, 12.0, 120, 13
    eps = si.guess_pulses(N, nt, T, 30.0)
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, si.shape_functions(N, nt, T), np.full(N, 10.0),
                 si.uniforms(9, 4, M, 9), precision=precision,
                 psi0_batch=si.random_states(109, M, (3 * (nc + 1)) ** N)) as p:
        p.update(3)
        nu = p.pulse_noise()
        nu_upd = p.pulse_noise(ref=eps)
        pulse = p.pulses()
    tol = 16 * np.finfo(float).eps * np.abs(pulse).max() * T
    want = noise.pulse_noise(pulse, T / nt)
    want_upd = noise.pulse_noise(pulse - eps, T / nt)
    assert np.all(want > 0) and np.all(want_upd > 0)
    np.testing.assert_allclose(nu, want, rtol=0, atol=tol)
    np.testing.assert_allclose(nu_upd, want_upd, rtol=0, atol=tol)
