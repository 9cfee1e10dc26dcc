"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics (CPU only).

Each test checks the oracle against something other than itself: closed forms, the paper's
printed effective model, an independent ODE solver, a library root finder, the density-matrix
solution, finite differences, invariants.  A plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.optimize
import scipy.sparse.linalg as spla

import synth_inputs as si
from oracle import gradient as og
from oracle import lindblad as ol
from oracle import mcwf
from oracle import model as om
from oracle.propagate import ChebyshevPropagator, StepPropagator, expm_propagator

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def cfg1_model(**kw):
    return om.build_model(2, 1, **kw)


# ---------------------------------------------------------------- model structure (Sec. 3.1)

def test_hermiticity_and_dissipator():
    m = cfg1_model()
    eps = np.array([0.7, -1.3])
    H = m.H(eps)
    assert np.abs(H - H.conj().T).max() == 0.0
    for hc in m.Hc:
        assert np.abs(hc - hc.conj().T).max() == 0.0
    Heff = m.Heff(eps)
    herm = 0.5 * (Heff + Heff.conj().T)
    anti = 0.5j * (Heff - Heff.conj().T)      # = +(1/2) L^dag L for H_eff = H - (i/2) L^dag L
    np.testing.assert_allclose(herm, H, atol=1e-14)
    np.testing.assert_allclose(anti, 0.5 * m.LdagL(), atol=1e-14)
    w = np.linalg.eigvalsh(m.LdagL())
    assert w.min() > -1e-12


def test_cascade_is_strictly_downstream():
    """H_int + (-(i/2) L^dag L) cancels every upstream hop a_i^dag a_j (i < j) exactly and
    leaves -2 i kappa a_j^dag a_i (photon from node i to node j > i)."""
    kappa = 0.7
    m = om.build_model(3, 1, kappa=kappa)
    Heff = m.Heff(np.zeros(3))
    # |g,1> on node i and |g,0> elsewhere  ->  |g,1> on node j
    for i in range(3):
        for j in range(i + 1, 3):
            photons_i = [0, 0, 0]; photons_i[i] = 1
            photons_j = [0, 0, 0]; photons_j[j] = 1
            xi = om.basis_index(1, [om.G] * 3, photons_i)
            xj = om.basis_index(1, [om.G] * 3, photons_j)
            assert Heff[xi, xj] == 0.0                          # no upstream coupling
            assert Heff[xj, xi] == pytest.approx(-2j * kappa)   # downstream coupling


def test_excitation_number_conserved_and_lowered_by_jumps():
    for (N, nc) in [(2, 1), (2, 2), (3, 1)]:
        m = om.build_model(N, nc)
        nexc = om.excitation_number(N, nc)
        H = m.H(np.random.default_rng(1).normal(size=N))
        comm = H * nexc[None, :] - nexc[:, None] * H
        assert np.abs(comm).max() < 1e-12
        rows, cols = np.nonzero(m.L[0])
        assert np.all(nexc[rows] == nexc[cols] - 1)


def test_adiabatic_elimination_reproduces_papers_effective_node():
    """For large Delta the three-level node restricted to {g, e} (x) cavity follows the
    paper's effective node Hamiltonian H_0 + H_d (Sec. 3.1), plus the laser light shift
    Omega^2/(4 Delta) on e that the same second-order elimination produces.  The error
    shrinks like 1/Delta.  Complex amplitudes are compared, so coupling phases are pinned."""
    n_cav, g, omega = 1, 1.0, 2.0
    nl = 3 * (n_cav + 1)

    def run(delta, t_end):
        m = om.build_model(1, n_cav, delta=delta, g=g, kappa=0.0)
        H3 = m.H(np.array([omega]))
        keep = [a * (n_cav + 1) + n for a in (om.G, om.E) for n in range(n_cav + 1)]
        # paper's effective node (Sec. 3.1): written out in the {g,e} (x) cavity basis
        a = om.cavity_lowering(n_cav)
        ad = a.conj().T
        Pg = np.diag([1.0, 0.0]).astype(complex)
        Pe = np.diag([0.0, 1.0]).astype(complex)
        s_eg = np.array([[0, 0], [1, 0]], dtype=complex)     # |e><g|
        Heff2 = (-(g * g / delta) * np.kron(np.eye(2), ad @ a)
                 + (g * g / delta) * np.kron(Pg, ad @ a)
                 - (1j * omega * g / (2 * delta)) * (np.kron(s_eg, a) - np.kron(s_eg, a).conj().T)
                 + (omega ** 2 / (4 * delta)) * np.kron(Pe, np.eye(n_cav + 1)))
        psi3 = np.zeros(nl, dtype=complex)
        psi3[om.G * (n_cav + 1) + 1] = 1.0           # |g, 1>
        psi2 = np.zeros(2 * (n_cav + 1), dtype=complex)
        psi2[1] = 1.0
        err = 0.0
        for t in np.linspace(0, t_end, 7)[1:]:
            a3 = expm_propagator(H3, t) @ psi3
            a2 = expm_propagator(Heff2, t) @ psi2
            err = max(err, np.abs(a3[keep] - a2).max())
        return err

    t_rabi = lambda delta: math.pi * delta / (omega * g)     # effective coupling Omega g / 2 Delta
    e1 = run(100.0, t_rabi(100.0))
    e2 = run(400.0, t_rabi(400.0))
    assert e1 < 0.05
    assert e2 < e1 / 3.0


# ---------------------------------------------------------------- propagators

@pytest.mark.parametrize("N,nc", [(2, 1), (2, 2)])
def test_chebyshev_matches_expm(N, nc):
    m = om.build_model(N, nc)
    Heff = m.Heff(np.array([1.3, -0.4]))
    cheb = ChebyshevPropagator(Heff)
    v = si.random_states(3, 5, m.d).T
    for tau in (0.1, 0.05, 0.013, 1e-7):
        ref = expm_propagator(Heff, tau) @ v
        np.testing.assert_allclose(cheb.apply(v, tau), ref, rtol=0, atol=1e-13)


def test_chebyshev_large_d_matches_expm_multiply():
    m = om.build_model(3, 2, kappa=1.0)
    import scipy.sparse as sp
    Heff = sp.csr_matrix(m.Heff(np.array([0.5, 1.0, -0.2])))
    v = si.random_states(4, 2, m.d).T
    ref = spla.expm_multiply(-1j * 0.025 * Heff, v)
    got = StepPropagator(Heff).apply(v, 0.025)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- special cases

def test_kappa_zero_is_norm_preserving_schroedinger():
    """kappa = 0: H_eff Hermitian, norm conserved, no jumps, and the trajectory equals the
    Schroedinger solution from an independent ODE integrator."""
    wl = si.CONFIGS["cfg1_d36"].with_(kappa=0.0, guess_amp=30.0, nt=100, T=10.0, M=3)
    m = om.build_model(2, 1, kappa=0.0)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    U = si.uniforms(7, 1, wl.M, wl.draws_per_traj)
    psi0 = si.random_states(8, wl.M, m.d)
    fw = mcwf.forward_pass(m, eps, wl.T, U[0], psi0, keep_states=True)
    assert sum(len(r) for r in fw.records) == 0
    norms = np.sum(np.abs(fw.psi_t) ** 2, axis=2)
    assert np.abs(norms - 1.0).max() < 1e-13
    dt = wl.dt
    y = psi0[0].copy()
    for j in range(wl.nt):
        H = m.H(eps[:, j])
        sol = scipy.integrate.solve_ivp(lambda t, x: -1j * (H @ x), (0, dt), y, method="DOP853",
                                        rtol=1e-13, atol=1e-14)
        y = sol.y[:, -1]
    assert np.abs(y - fw.psi_T[0]).max() < 1e-9


def test_zero_pulse_is_stationary():
    """eps = 0: |e g..g, 0..0> is an exact zero-energy eigenstate of H_eff, so psi(t) = psi0,
    F = 1/N, no jumps and the Krotov update vanishes identically."""
    for (N, nc) in [(2, 1), (3, 1)]:
        m = om.build_model(N, nc)
        nt, T, M = 40, 4.0, 4
        eps = np.zeros((N, nt))
        U = si.uniforms(1, 2, M, 1 + 2 * N * (1 + nc))
        S = si.shape_functions(N, nt, T)
        res = mcwf.optimize(m, eps, T, U, S, np.full(N, 10.0), 1, keep=True)
        fw = res.forward[-1]
        np.testing.assert_allclose(fw.psi_T, np.broadcast_to(m.psi0, fw.psi_T.shape), atol=1e-14)
        assert res.JT[0] == pytest.approx(1.0 - 1.0 / N, abs=1e-14)
        assert np.abs(fw.deps).max() == 0.0
        assert sum(len(r) for r in fw.records) == 0


def test_single_cavity_decay_jump_time_closed_form():
    """One node with g = 0 started in |g,1>: an eigenvector of H_eff with eigenvalue -i kappa,
    so ||psi(t)||^2 = exp(-2 kappa t) and the jump happens at t* = -ln(r) / (2 kappa)."""
    kappa = 0.8
    m = om.build_model(1, 1, g=0.0, kappa=kappa)
    psi0 = np.zeros(m.d, dtype=complex)
    psi0[om.basis_index(1, [om.G], [1])] = 1.0
    T, nt, M = 4.0, 40, 16
    U = si.uniforms(11, 1, M, 3)
    fw = mcwf.forward_pass(m, np.zeros((1, nt)), T, U[0], psi0)
    dt = T / nt
    for k in range(M):
        t_star = -math.log(U[0, k, 0]) / (2 * kappa)
        if t_star < T:
            assert len(fw.records[k]) == 1
            rec = fw.records[k][0]
            assert abs((rec.step - 1) * dt + rec.s - t_star) < 1e-11 * dt + 1e-14
            assert rec.c == pytest.approx(1.0 / math.sqrt(2 * kappa * math.exp(-2 * kappa * t_star)), rel=1e-9)
        else:
            assert len(fw.records[k]) == 0


def test_jump_times_match_brute_force_no_jump_norm():
    """Paper's initial state has one excitation, so at most one jump.  The jump time is the
    first root of ||psi_nojump(t)||^2 = r, found here by scanning the no-jump norm and
    refining with brentq (independent of the oracle's bisection).  A jumped trajectory ends
    in |g..g, 0..0> with fidelity 0 ("a total loss", Sec. 3.3)."""
    wl = si.CONFIGS["cfg1_d36"].with_(guess_amp=30.0)
    m = om.build_model(2, 1)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    U = si.uniforms(wl.seed, 1, wl.M, wl.draws_per_traj)
    fw = mcwf.forward_pass(m, eps, wl.T, U[0], m.psi0)
    dt = wl.dt
    # no-jump norm curve on the grid
    psi = m.psi0.copy()
    norms = [1.0]
    states = [psi]
    for j in range(wl.nt):
        psi = expm_propagator(m.Heff(eps[:, j]), dt) @ psi
        states.append(psi)
        norms.append(float(np.vdot(psi, psi).real))
    norms = np.array(norms)
    n_jumped = 0
    for k in range(wl.M):
        r = U[0, k, 0]
        below = np.nonzero(norms <= r)[0]
        if len(below) == 0:
            assert fw.records[k] == []
            continue
        j = int(below[0])            # interval j holds the crossing
        Hj = m.Heff(eps[:, j - 1])
        f = lambda s: float(np.linalg.norm(expm_propagator(Hj, s) @ states[j - 1]) ** 2) - r
        s_ref = scipy.optimize.brentq(f, 0.0, dt, xtol=1e-15, rtol=1e-15)
        assert len(fw.records[k]) == 1
        rec = fw.records[k][0]
        assert rec.step == j
        assert abs(rec.s - s_ref) < 1e-9 * dt
        n_jumped += 1
        ground = np.zeros(m.d); ground[0] = 1.0
        phat = fw.psi_T[k] / np.linalg.norm(fw.psi_T[k])
        assert abs(abs(np.vdot(ground, phat)) - 1.0) < 1e-12
        assert abs(np.vdot(m.psi_tgt, phat)) < 1e-14
    assert n_jumped >= 5


def test_excitation_sector_stays_exactly_empty():
    wl = si.CONFIGS["cfg1_d36"].with_(guess_amp=30.0, nt=200, T=20.0, M=16)
    m = om.build_model(2, 1)
    nexc = om.excitation_number(2, 1)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    U = si.uniforms(3, 1, wl.M, wl.draws_per_traj)
    fw = mcwf.forward_pass(m, eps, wl.T, U[0], m.psi0, keep_states=True)
    outside = fw.psi_t[:, :, nexc > 1]
    assert np.abs(outside).max() == 0.0


# ---------------------------------------------------------------- statistics (Eq. rho_traj_expansion)

@pytest.mark.slow
def test_trajectory_average_converges_to_lindblad():
    """|mean_k |tau_k|^2 - <tgt|rho(T)|tgt>| <= 3 sigma / sqrt(M), and the jump fraction
    equals 1 - ||psi_nojump(T)||^2 within the binomial 3 sigma."""
    T, nt, M = 20.0, 200, 2048
    m = om.build_model(2, 1)
    eps = si.guess_pulses(2, nt, T, 40.0)
    U = si.uniforms(21, 1, M, 5)
    fw = mcwf.forward_pass(m, eps, T, U[0], m.psi0)
    tau, F = mcwf.fidelity(fw.psi_T, m.psi_tgt)
    rho0 = np.outer(m.psi0, m.psi0.conj())
    rho = ol.propagate_rho(m, eps, T, rho0)
    assert abs(np.trace(rho) - 1.0) < 1e-10
    f_rho = float(np.vdot(m.psi_tgt, rho @ m.psi_tgt).real)
    sigma = np.std(np.abs(tau) ** 2)
    assert abs(F - f_rho) <= 3 * sigma / math.sqrt(M)
    psi = m.psi0.copy()
    for j in range(nt):
        psi = expm_propagator(m.Heff(eps[:, j]), T / nt) @ psi
    p_jump = 1.0 - float(np.vdot(psi, psi).real)
    frac = np.mean([len(r) > 0 for r in fw.records])
    assert 0.05 < p_jump < 0.95
    assert abs(frac - p_jump) <= 3 * math.sqrt(p_jump * (1 - p_jump) / M)


def test_lindblad_single_cavity_decay_closed_form():
    kappa = 0.6
    a = om.cavity_lowering(2)
    class Cav:
        L = [math.sqrt(2 * kappa) * a]
        def Heff(self, eps):
            return -0.5j * self.L[0].conj().T @ self.L[0]
    rho0 = np.zeros((3, 3), dtype=complex); rho0[2, 2] = 1.0
    T = 1.3
    rho = ol.propagate_rho(Cav(), np.zeros((1, 13)), T, rho0)
    p2 = math.exp(-4 * kappa * T)
    p1 = 2 * math.exp(-2 * kappa * T) * (1 - math.exp(-2 * kappa * T))
    assert rho[2, 2].real == pytest.approx(p2, abs=1e-12)
    assert rho[1, 1].real == pytest.approx(p1, abs=1e-12)
    assert np.trace(rho).real == pytest.approx(1.0, abs=1e-12)


# ---------------------------------------------------------------- backward sweep and update

def test_backward_sweep_is_the_adjoint_of_the_forward_map():
    """With the same pulse and record, <chi_k(t_j)|psi_k(t_j)> is the same at every t_j."""
    wl = si.CONFIGS["cfg1_d36"].with_(guess_amp=30.0, nt=120, T=12.0, M=12)
    m = om.build_model(2, 1)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    U = si.uniforms(9, 1, wl.M, wl.draws_per_traj)
    psi0 = si.random_states(10, wl.M, m.d)
    fw = mcwf.forward_pass(m, eps, wl.T, U[0], psi0, keep_states=True)
    assert sum(len(r) for r in fw.records) >= 3
    chi_T = si.random_states(12, wl.M, m.d)
    chi = mcwf.backward_pass(m, eps, wl.T, chi_T, fw.records)
    ov = np.einsum("tkd,tkd->tk", chi.conj(), fw.psi_t)
    assert np.abs(ov - ov[-1][None, :]).max() < 1e-12


def test_first_interval_update_is_the_first_order_gradient():
    """At j = 1 (psi^(1)(t_0) = psi^(0)(t_0)) the update equals -S/(2 lambda dt) dJ_T/deps_1
    to first order in dt (Eq. independent_traj_update vs Eq. gradient); the relative gap
    shrinks linearly as dt -> 0 (kappa = 0, one trajectory, no jumps)."""
    m = om.build_model(2, 1, delta=5.0, kappa=0.0)
    lam = np.array([10.0, 10.0])
    gaps = []
    for nt in (400, 800):
        T = 4.0
        dt = T / nt
        eps = si.guess_pulses(2, nt, T, 3.0) + 0.3
        S = np.ones((2, nt))
        U = si.uniforms(0, 2, 1, 5)
        fw0 = mcwf.forward_pass(m, eps, T, U[0], m.psi0)
        tau, _ = mcwf.fidelity(fw0.psi_T, m.psi_tgt)
        chi = mcwf.backward_pass(m, eps, T, tau[:, None] * m.psi_tgt[None, :], fw0.records)
        fw1 = mcwf.forward_pass(m, eps, T, U[1], m.psi0, chi=chi, shape=S, lam=lam)
        h = 1e-5
        grad0 = np.zeros(2)
        for i in range(2):
            ep = eps.copy(); ep[i, 0] += h
            em = eps.copy(); em[i, 0] -= h
            Fp = mcwf.fidelity(mcwf.forward_pass(m, ep, T, U[0], m.psi0).psi_T, m.psi_tgt)[1]
            Fm = mcwf.fidelity(mcwf.forward_pass(m, em, T, U[0], m.psi0).psi_T, m.psi_tgt)[1]
            grad0[i] = -(Fp - Fm) / (2 * h)
        pred = -S[:, 0] / (2 * lam * dt) * grad0
        gaps.append(np.abs(fw1.deps[:, 0] - pred).max() / np.abs(pred).max())
    assert gaps[0] < 0.02
    assert gaps[1] < 0.6 * gaps[0]


def test_krotov_monotone_at_kappa_zero():
    """Deterministic case (kappa = 0, one trajectory): J_T decreases at every iteration."""
    wl = si.CONFIGS["cfg1_d36"].with_(kappa=0.0, guess_amp=30.0, nt=200, T=20.0, M=1)
    m = om.build_model(2, 1, kappa=0.0)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    S = si.shape_functions(2, wl.nt, wl.T)
    U = si.uniforms(0, 9, 1, wl.draws_per_traj)
    res = mcwf.optimize(m, eps, wl.T, U, S, np.full(2, 0.2), 8)
    JT = np.array(res.JT)
    assert np.all(np.diff(JT) < 0.0)
    assert JT[-1] < JT[0] - 5e-4


# ---------------------------------------------------------------- gradient (frozen record)

def test_gradient_matches_finite_differences_with_jumps():
    wl = si.CONFIGS["cfg1_d36"].with_(guess_amp=30.0, nt=60, T=6.0, M=6)
    m = om.build_model(2, 1)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    U = si.uniforms(5, 1, wl.M, wl.draws_per_traj)
    psi0 = si.random_states(6, wl.M, m.d)
    fw = mcwf.forward_pass(m, eps, wl.T, U[0], psi0)
    assert sum(len(r) for r in fw.records) >= 2
    grad, jt = og.gradient(m, eps, wl.T, psi0, fw.records)
    _, F = mcwf.fidelity(fw.psi_T, m.psi_tgt)
    assert jt == pytest.approx(1.0 - F, abs=1e-13)
    rng = np.random.default_rng(0)
    slots = [(int(rng.integers(2)), int(rng.integers(wl.nt))) for _ in range(10)]
    fd = og.fd_gradient(m, eps, wl.T, psi0, fw.records, slots, h=1e-4)
    ref = np.array([grad[i, j] for i, j in slots])
    assert np.abs(fd - ref).max() <= 1e-6 * np.abs(ref).max() + 1e-11


def test_gradient_matches_free_running_fd_at_kappa_zero():
    wl = si.CONFIGS["cfg1_d36"].with_(kappa=0.0, guess_amp=30.0, nt=50, T=5.0, M=2)
    m = om.build_model(2, 1, kappa=0.0)
    eps = si.guess_pulses(2, wl.nt, wl.T, wl.guess_amp)
    U = si.uniforms(5, 1, wl.M, wl.draws_per_traj)
    psi0 = si.random_states(2, wl.M, m.d)
    fw = mcwf.forward_pass(m, eps, wl.T, U[0], psi0)
    grad, _ = og.gradient(m, eps, wl.T, psi0, fw.records)
    h = 1e-4
    for (i, j) in [(0, 3), (1, 25), (0, 49)]:
        ep = eps.copy(); ep[i, j] += h
        em = eps.copy(); em[i, j] -= h
        Fp = mcwf.fidelity(mcwf.forward_pass(m, ep, wl.T, U[0], psi0).psi_T, m.psi_tgt)[1]
        Fm = mcwf.fidelity(mcwf.forward_pass(m, em, wl.T, U[0], psi0).psi_T, m.psi_tgt)[1]
        fd = -(Fp - Fm) / (2 * h)
        assert fd == pytest.approx(grad[i, j], rel=1e-6, abs=1e-11)


# ---------------------------------------------------------------- noise measure (Eq. noise)
def test_savitzky_golay_reproduces_cubics_and_published_weights():
    """A cubic least-squares smoother leaves any cubic unchanged (nu = 0), and its centred
    five-point weights are the published convolute (-3, 12, 17, 12, -3)/35."""
    from oracle import noise
    t = np.linspace(-1.0, 2.0, 40)
    cubic = 0.3 - 1.2 * t + 0.7 * t ** 2 + 0.25 * t ** 3
    np.testing.assert_allclose(noise.savitzky_golay_cubic5(cubic), cubic, rtol=0, atol=1e-12)
    assert noise.pulse_noise(cubic[None, :], 0.1)[0] <= 1e-11
    for k in range(5):
        e = np.zeros(11)
        e[3 + k] = 1.0
        assert noise.savitzky_golay_cubic5(e)[5] == pytest.approx([-3, 12, 17, 12, -3][4 - k] / 35.0, abs=1e-14)


def test_savitzky_golay_matches_scipy_interp_mode():
    from scipy.signal import savgol_filter
    from oracle import noise
    y = np.random.default_rng(3).normal(size=57)
    np.testing.assert_allclose(noise.savitzky_golay_cubic5(y), savgol_filter(y, 5, 3, mode="interp"),
                               rtol=0, atol=1e-12)


def test_noise_of_white_noise_scales_and_power_law_fit():
    """nu is linear in the noise amplitude and the log-log fit recovers an exact power law."""
    from oracle import noise
    rng = np.random.default_rng(4)
    base = np.sin(np.linspace(0, np.pi, 400)) ** 2
    w = rng.normal(size=400)
    n1 = noise.pulse_noise((base + 1e-3 * w)[None, :], 0.05)[0]
    n2 = noise.pulse_noise((base + 2e-3 * w)[None, :], 0.05)[0]
    assert n2 / n1 == pytest.approx(2.0, rel=1e-3)
    M = np.array([4, 16, 64, 256])
    assert noise.fit_power_law(M, 3.0 / np.sqrt(M)) == pytest.approx(-0.5, abs=1e-12)


# ---------------------------------------------------------------- cross-trajectory update
def test_cross_overlap_is_the_trace_of_the_two_projectors():
    """sum_{k,k'} <xi_k|H|psi_k'><psi_k'|xi_k> = tr(H R Pi) with R = sum |psi><psi|, Pi = sum |xi><xi|:
    fixes which factor carries k and which k' (a transposed operand changes the value)."""
    rng = np.random.default_rng(11)
    M, d = 5, 7
    xi = rng.normal(size=(M, d)) + 1j * rng.normal(size=(M, d))
    psi = rng.normal(size=(M, d)) + 1j * rng.normal(size=(M, d))
    H = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    H = H + H.conj().T
    R = sum(np.outer(p, p.conj()) for p in psi)
    Pi = sum(np.outer(x, x.conj()) for x in xi)
    assert mcwf.cross_overlap(xi, psi, H) == pytest.approx(np.imag(np.trace(H @ R @ Pi)), rel=1e-12)
    swapped = float(np.sum(np.imag((np.conj(xi) @ (psi @ H.T).T).T * np.conj(np.conj(xi) @ psi.T))))
    assert abs(swapped - np.imag(np.trace(H @ R @ Pi))) > 1e-3


def test_cross_update_equals_independent_for_one_closed_trajectory_at_t0():
    """M = 1, kappa = 0: <psi(t_0)|xi(t_0)> = <psi(T)|tgt> = conj(tau) (norm 1), so the first
    interval's cross update equals the independent one; later intervals differ."""
    m = om.build_model(2, 1, kappa=0.0)
    nt, T = 30, 3.0
    eps = si.guess_pulses(2, nt, T, 20.0)
    S = si.shape_functions(2, nt, T)
    lam = np.full(2, 10.0)
    U = si.uniforms(0, 2, 1, 9)
    a = mcwf.optimize(m, eps, T, U, S, lam, 1, keep=True)
    b = mcwf.optimize(m, eps, T, U, S, lam, 1, keep=True, update="cross")
    da, db = a.forward[1].deps, b.forward[1].deps
    assert np.abs(da[:, 0]).max() > 1e-8
    np.testing.assert_allclose(db[:, 0], da[:, 0], rtol=1e-10, atol=1e-18)
    assert np.abs(db - da).max() > 1e-6 * np.abs(da).max()


# ---------------------------------------------------------------- first-order jump scheme
def test_first_order_jump_lands_at_the_end_of_the_interval_containing_the_exact_time():
    """Same decaying cavity as the closed-form pin: with at most one jump per step, decided at the
    end of the step, the jump of trajectory k is recorded in interval ceil(t*/dt) at s* = dt, with
    c = 1/||L psi(t_j)|| = 1/sqrt(2 kappa exp(-2 kappa t_j))."""
    kappa = 0.8
    m = om.build_model(1, 1, g=0.0, kappa=kappa)
    psi0 = np.zeros(m.d, dtype=complex)
    psi0[om.basis_index(1, [om.G], [1])] = 1.0
    T, nt, M = 4.0, 40, 16
    U = si.uniforms(11, 1, M, 3)
    fw = mcwf.forward_pass(m, np.zeros((1, nt)), T, U[0], psi0, first_order=True)
    dt = T / nt
    n_jumped = 0
    for k in range(M):
        t_star = -math.log(U[0, k, 0]) / (2 * kappa)
        j = math.ceil(t_star / dt)
        if j <= nt:
            n_jumped += 1
            assert len(fw.records[k]) == 1
            rec = fw.records[k][0]
            assert rec.step == j and rec.s == dt
            assert rec.c == pytest.approx(1.0 / math.sqrt(2 * kappa * math.exp(-2 * kappa * j * dt)), rel=1e-9)
        else:
            assert len(fw.records[k]) == 0
    assert n_jumped >= 5


def test_complex_coupling_is_a_photon_number_gauge_of_the_real_one():
    """With g = |g| e^{i phi}, H_eff = V H_eff(|g|) V^dag for V = exp(-i phi N_phot) (N_phot the
    total photon number): the phase only rotates a, which the cascade hops a_j^dag a_i, L^dag L
    and the drive do not see.  A dropped conjugate or a wrong |g|^2 breaks the identity."""
    phi = 0.7
    gc = 1.3 * complex(math.cos(phi), math.sin(phi))
    mc = om.build_model(2, 2, g=gc)
    mr = om.build_model(2, 2, g=1.3)
    nl, NP = 9, 3
    x = np.arange(nl * nl)
    nph = (x // nl) % NP + (x % nl) % NP          # local index = atom * (n_cav + 1) + n
    V = np.diag(np.exp(-1j * phi * nph))
    eps = np.array([0.4, -0.9])
    Hc, Hr = mc.Heff(eps), mr.Heff(eps)
    np.testing.assert_allclose(Hc, V @ Hr @ V.conj().T, rtol=0, atol=1e-12 * np.abs(Hr).max())
    assert np.abs(Hc - Hr).max() > 0.1                # the phase is really there


# ---------------------------------------------------------------- density-matrix Krotov
def test_density_backward_map_is_the_adjoint():
    """<<P(t_j)|rho(t_j)>> is the same at every t_j under one pulse (fixes E^dag, not E^T or E)."""
    from oracle import density as od
    m = om.build_model(1, 1)
    nt, T = 12, 3.0
    eps = si.guess_pulses(1, nt, T, 20.0)
    rho = ol.propagate_rho(m, eps, T, np.outer(m.psi0, m.psi0.conj()), dense=True, keep=True)
    P = od.backward_P(m, eps, T, np.outer(m.psi_tgt, m.psi_tgt.conj()))
    pair = [np.trace(P[j].conj().T @ rho[j]) for j in range(nt + 1)]
    np.testing.assert_allclose(pair, pair[-1], rtol=1e-11, atol=1e-13)


def test_density_update_is_the_first_order_descent_direction():
    """Delta u_1 = -S / (lambda dt) dJ_T/du_1 to first order in dt (central differences of J_T
    from the density-matrix propagation): fixes the sign and the factor of Eq. krotovupdate with
    dL/du rho = [H, rho] and dE/du = -i dt [H, .] to first order."""
    from oracle import density as od
    m = om.build_model(1, 1)
    nt, T = 400, 4.0
    dt = T / nt
    eps = si.guess_pulses(1, nt, T, 20.0)
    S = np.ones((1, nt))
    lam = np.array([2.0])
    rho0 = np.outer(m.psi0, m.psi0.conj())
    P = od.backward_P(m, eps, T, np.outer(m.psi_tgt, m.psi_tgt.conj()))
    _, deps, _ = od.forward_update(m, eps, T, rho0, P, S, lam)
    h = 1e-5
    ep, em = eps.copy(), eps.copy()
    ep[0, 0] += h
    em[0, 0] -= h
    Jp = od.functional(m, ol.propagate_rho(m, ep, T, rho0, dense=True))
    Jm = od.functional(m, ol.propagate_rho(m, em, T, rho0, dense=True))
    grad = (Jp - Jm) / (2 * h)
    assert abs(grad) > 1e-8
    assert deps[0, 0] == pytest.approx(-S[0, 0] / (lam[0] * dt) * grad, rel=2e-2)


def test_density_update_is_twice_the_trajectory_update_for_a_closed_pure_state():
    """kappa = 0, pure initial state: P(t) = |xi><xi|, rho = |psi><psi|, and Im<<P|[H, rho]>> =
    2 Im[<xi|H|psi><psi|xi>] = 2 Im<chi|H|psi> at t_0 (chi = tau xi, <psi_0|xi(t_0)> = conj(tau));
    so the first interval's density-matrix update is twice the one-trajectory update."""
    from oracle import density as od
    m = om.build_model(1, 1, kappa=0.0)
    nt, T = 40, 4.0
    eps = si.guess_pulses(1, nt, T, 20.0)
    S = si.shape_functions(1, nt, T)
    lam = np.full(1, 10.0)
    psi0 = si.random_states(5, 1, m.d)[0]
    rho0 = np.outer(psi0, psi0.conj())
    P = od.backward_P(m, eps, T, np.outer(m.psi_tgt, m.psi_tgt.conj()))
    _, d_dm, _ = od.forward_update(m, eps, T, rho0, P, S, lam)
    res = mcwf.optimize(m, eps, T, si.uniforms(0, 2, 1, 5), S, lam, 1, psi0=psi0, keep=True)
    d_traj = res.forward[1].deps
    assert abs(d_traj[0, 0]) > 1e-10
    np.testing.assert_allclose(d_dm[:, 0], 2.0 * d_traj[:, 0], rtol=1e-8, atol=1e-16)


def test_density_krotov_is_monotone_with_dissipation():
    """The density-matrix functional is linear in rho and the dynamics linear in u, so first-order
    Krotov lowers J_T at every iteration, here with cavity decay (kappa = 1)."""
    from oracle import density as od
    m = om.build_model(1, 1)
    nt, T = 40, 4.0
    JT, _ = od.optimize_dm(m, si.guess_pulses(1, nt, T, 20.0), T, si.shape_functions(1, nt, T), np.array([5.0]), 4)
    assert np.all(np.diff(JT) < 0.0)


# ---------------------------------------------------------------- Krotov's functional, channels, large-d adjoint
def test_krotov_functional_is_stationary_at_the_first_interval_update():
    """Krotov's update minimises J = J_T + sum_i lambda_i/S_i int Delta eps_i^2 dt (Eq.
    krotov_functional) to first order: f(D) = J(eps + D e_i1) with the penalty of that one
    interval is stationary at D = the oracle's Delta eps_i1 up to O(dt) (kappa = 0, one
    trajectory, S != 1 and lambda differing between the controls).  f'(D) = dJ_T/deps_i1 +
    2 lambda_i D dt / S_i: a penalty with lambda S, S / lambda, without dt or linear in D leaves a
    derivative of the size of dJ_T/deps itself, or far larger.  The gap shrinks as dt -> 0."""
    m = om.build_model(2, 1, delta=5.0, kappa=0.0)
    lam = np.array([10.0, 3.0])
    ratios = []
    for nt in (400, 800):
        T = 4.0
        dt = T / nt
        eps = si.guess_pulses(2, nt, T, 3.0) + 0.3
        S = np.empty((2, nt))
        S[0], S[1] = 0.37, 0.8
        U = si.uniforms(0, 2, 1, 5)
        psi0 = si.random_states(3, 1, m.d)[0]     # both nodes driven at t_0: both updates nonzero
        fw0 = mcwf.forward_pass(m, eps, T, U[0], psi0)
        tau, _ = mcwf.fidelity(fw0.psi_T, m.psi_tgt)
        chi = mcwf.backward_pass(m, eps, T, tau[:, None] * m.psi_tgt[None, :], fw0.records)
        fw1 = mcwf.forward_pass(m, eps, T, U[1], psi0, chi=chi, shape=S, lam=lam)
        worst = 0.0
        for i in range(2):
            d_star = fw1.deps[i, 0]
            assert abs(d_star) > 1e-9
            h = 1e-4 * abs(d_star)

            def f(D):
                ep = eps.copy()
                ep[i, 0] += D
                JT = 1.0 - mcwf.fidelity(mcwf.forward_pass(m, ep, T, U[0], psi0).psi_T, m.psi_tgt)[1]
                dmat = np.zeros_like(eps)
                dmat[i, 0] = D
                return mcwf.krotov_functional(JT, dmat, S, lam, dt)

            slope = (f(d_star + h) - f(d_star - h)) / (2 * h)
            # dJ_T/deps_i1 = -2 lambda_i D* dt / S_i at the stationary point: the scale of each term
            scale = 2 * lam[i] * abs(d_star) * dt / S[i, 0]
            worst = max(worst, abs(slope) / scale)
        ratios.append(worst)
    # measured 0.074 -> 0.037; lambda S in place of lambda / S stays near 0.8, no dt gives ~1e2
    assert ratios[0] < 0.15
    assert ratios[1] < 0.6 * ratios[0]


def test_channel_choice_matches_integrated_channel_rates():
    """Several Lindblad operators (Sec. 2.1: the jump goes to channel l with probability
    proportional to <psi|L_l^dag L_l|psi>).  Two cavity modes coupled by the cascade hop
    i kappa (a_0^dag a_1 - a_1^dag a_0), one photon shared as alpha |1,0> + beta |0,1>, atoms
    decoupled (g = 0, eps = 0), one detector per cavity L_l = sqrt(2 kappa) a_l: the no-jump
    amplitudes are c(t) = exp(-kappa t) R(kappa t) c(0) with R a rotation, and channel l fires
    with total probability 2 kappa int_0^inf |c_l(t)|^2 dt = (3 alpha^2 + 2 alpha beta + beta^2)/4
    for l = 0 (the rest for l = 1).  The chosen channels' frequency over 1500 trajectories
    matches within the binomial 3 sigma; choosing the other channel, or by u alone, fails."""
    m = om.build_model(2, 1, g=0.0, kappa=1.0, lindblad="local")
    assert len(m.L) == 2
    a2 = 0.3
    al, be = math.sqrt(a2), math.sqrt(1.0 - a2)
    psi0 = np.zeros(m.d, dtype=np.complex128)
    psi0[om.basis_index(1, [0, 0], [1, 0])] = al
    psi0[om.basis_index(1, [0, 0], [0, 1])] = be
    M, nt, T = 1500, 40, 8.0                      # exp(-2 kappa T) ~ 1e-7: every trajectory jumps once
    U = si.uniforms(21, 1, M, 5)
    fw = mcwf.forward_pass(m, np.zeros((2, nt)), T, U[0], psi0)
    assert all(len(r) == 1 for r in fw.records)
    p0 = (3 * a2 + 2 * al * be + (1 - a2)) / 4
    freq = np.mean([r[0].channel == 0 for r in fw.records])
    assert abs(freq - p0) <= 3 * math.sqrt(p0 * (1 - p0) / M), (freq, p0)


def test_backward_sweep_is_the_adjoint_at_d729():
    """The pathwise co-state sweep on the three-node chain (d = 729), where the oracle propagates
    with its Chebyshev series on -H_eff^dag instead of expm: <chi_k(t_j)|psi_k(t_j)> is the same
    at every t_j along trajectories with jumps."""
    m = om.build_model(3, 2)
    nt, T, M = 20, 0.5, 3
    eps = si.guess_pulses(3, nt, T, 30.0)
    U = si.uniforms(2, 1, M, 1 + 2 * 9)
    psi0 = si.random_states(102, M, m.d)
    fw = mcwf.forward_pass(m, eps, T, U[0], psi0, keep_states=True)
    assert sum(len(r) for r in fw.records) >= 1
    chi_T = si.random_states(12, M, m.d)
    chi = mcwf.backward_pass(m, eps, T, chi_T, fw.records)
    ov = np.einsum("tkd,tkd->tk", chi.conj(), fw.psi_t)
    assert np.abs(ov - ov[-1][None, :]).max() < 1e-11
