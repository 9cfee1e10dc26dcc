"""Density-matrix Krotov on the GPU (Sec. 2.2, Eqs. krotov_functional, krotovupdate, krotov_boundary)
against the FP64 oracle ``oracle/density.py``.

The library propagates vec(rho) as one state of the 2N-node Liouville-space network with the
trajectory kernels (no jumps, no normalisation); P(t) runs backward under the adjoint dynamics from
P(T) = |tgt><tgt|, and the pulse is updated sequentially by S/lambda Im <<P|[H_c, rho]>>.
Tolerances: FP64 1e-10 (rho(T), P(t_j) relative to their largest entry, F, Delta eps relative to
max |Delta eps|); FP32-mixed: F within 1e-5, Delta eps within 1e-4 of max |Delta eps| (the
trajectory path's stated tolerances).
"""
import numpy as np
import pytest

import synth_inputs as si
from oracle import density as od
from oracle import lindblad as ol
from oracle import model as om
from paper_1801_04382_gb300 import DensityProblem, KrotovError, cascaded_chain

pytestmark = pytest.mark.gpu


def _case(N, nc, T, nt, amp, lind="collective"):
    net = cascaded_chain(N, nc, lindblad=lind)
    m = om.build_model(N, nc, lindblad=lind)
    eps0 = si.guess_pulses(N, nt, T, amp)
    S = si.shape_functions(N, nt, T)
    lam = np.full(N, 2.0)
    return net, m, eps0, S, lam


def _oracle_iteration(m, eps0, T, S, lam):
    rho0 = np.outer(m.psi0, m.psi0.conj())
    F0 = 1.0 - od.functional(m, ol.propagate_rho(m, eps0, T, rho0, dense=True))
    P = od.backward_P(m, eps0, T, np.outer(m.psi_tgt, m.psi_tgt.conj()))
    eps1, deps, rho_T = od.forward_update(m, eps0, T, rho0, P, S, lam)
    return F0, P, eps1, deps, rho_T, 1.0 - od.functional(m, rho_T)


@pytest.mark.parametrize("N,nc,T,nt,lind", [(1, 2, 4.0, 200, "collective"), (2, 1, 0.6, 6, "collective"),
                                            (2, 1, 0.6, 6, "local")])
def test_density_krotov_iteration_matches_oracle_fp64(N, nc, T, nt, lind):
    """Guess sweep, backward sweep and updating forward sweep of density-matrix Krotov: F, P(t_j),
    Delta eps, rho(T) at the FP64 tolerance (one node over 200 intervals; the two-node chain with
    its cascade, collective or per-node decay, over 6)."""
    net, m, eps0, S, lam = _case(N, nc, T, nt, 20.0, lind)
    F0, P, eps1, deps, rho_T, F1 = _oracle_iteration(m, eps0, T, S, lam)
    with DensityProblem(net, T, nt, eps0, S, lam) as p:
        assert p.info.d == m.d ** 2 and p.info.tile_traj == 1
        g0 = p.forward(False)
        p.backward()
        for j in sorted({0, 1, nt // 2, nt - 1, nt}):
            Pj = p.P(j)
            assert np.abs(Pj - P[j]).max() <= 1e-10 * np.abs(P[j]).max(), j
        g1 = p.forward(True)
        g_deps, g_eps, g_rho = p.deps(), p.pulses(), p.rho()
    assert abs(g0 - F0) <= 1e-10 and abs(g1 - F1) <= 1e-10, (g0, F0, g1, F1)
    dmax = np.abs(deps).max()
    assert dmax > 0.0
    assert np.abs(g_deps - deps).max() <= 1e-10 * dmax
    assert np.abs(g_eps - eps1).max() <= 4e-10 * dmax
    assert np.abs(g_rho - rho_T).max() <= 1e-10 * np.abs(rho_T).max()


def test_density_krotov_is_monotone_on_the_gpu_and_matches_the_oracle_history():
    """Four density-matrix Krotov iterations with cavity decay through krotov_update (the graph
    path): J_T decreases at every iteration (first-order Krotov on a functional linear in rho) and
    equals the oracle's history at 1e-10."""
    net, m, eps0, S, lam = _case(1, 1, 4.0, 40, 20.0)
    lam = np.array([5.0])
    JT_ref, eps_ref = od.optimize_dm(m, eps0, 4.0, S, lam, 4)
    with DensityProblem(net, 4.0, 40, eps0, S, lam) as p:
        F0 = p.forward(False)
        JT, J = p.update(4)
        eps = p.pulses()
    assert abs((1.0 - F0) - JT_ref[0]) <= 1e-10
    np.testing.assert_allclose(JT, JT_ref[1:], rtol=0, atol=1e-10)
    assert np.all(np.diff(np.concatenate([[1.0 - F0], JT])) < 0.0)
    assert np.abs(eps - eps_ref).max() <= 1e-10 * np.abs(eps_ref).max()
    assert np.all(np.array(J) >= np.array(JT))


def test_density_krotov_fp32_mixed():
    """FP32-mixed Liouville-space propagation (complex64 vec(rho), FP64 overlaps and sums) against the
    FP64 oracle at the FP32 tolerances, co-states checkpointed every 7 intervals."""
    N, nc, T, nt = 1, 2, 4.0, 60
    net, m, eps0, S, lam = _case(N, nc, T, nt, 20.0)
    F0, P, eps1, deps, rho_T, F1 = _oracle_iteration(m, eps0, T, S, lam)
    with DensityProblem(net, T, nt, eps0, S, lam, precision="fp32", ckpt_interval=7) as p:
        g0 = p.forward(False)
        p.backward()
        g1 = p.forward(True)
        g_deps = p.deps()
    assert abs(g0 - F0) <= 1e-5 and abs(g1 - F1) <= 1e-5
    assert np.abs(g_deps - deps).max() <= 1e-4 * np.abs(deps).max()


def test_density_problem_refuses_the_trajectory_gradient():
    net, m, eps0, S, lam = _case(1, 1, 1.0, 10, 2.0)
    with DensityProblem(net, 1.0, 10, eps0, S, lam) as p:
        with pytest.raises(KrotovError, match="UNSUPPORTED"):
            p.forward(keep_for_gradient=True)
