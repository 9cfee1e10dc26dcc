"""Host-side checks of the C ABI library (no GPU needed): it loads, exports every symbol the
header declares, its Bessel helper matches SciPy, and descriptor validation rejects bad input
before any device call."""
import ctypes as ct
import os
import re

import numpy as np
import pytest
import scipy.special

import synth_inputs as si
from paper_1801_04382_gb300 import _capi, build as pkg_build, model as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg_build.lib_path()):
        pkg_build.build()
    return _capi.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "krotov_traj.h")).read()
    return set(re.findall(r"KT_API\s+[\w\s\*]+?\b(\w+)\s*\(", text))


def test_header_and_binding_agree(lib):
    syms = header_symbols()
    assert syms == set(_capi.SIGNATURES), syms ^ set(_capi.SIGNATURES)
    for name in syms:
        assert hasattr(lib, name), name


def test_exports_with_nm(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", pkg_build.lib_path()], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert header_symbols() <= exported


@pytest.mark.parametrize("alpha", [0.0, 1e-12, 1e-3, 0.37, 1.0, 2.2, 5.2, 9.9, 30.0])
def test_bessel_miller_matches_scipy(lib, alpha):
    n = 64
    out = np.zeros(n)
    assert lib.kt_bessel_j(alpha, n, out.ctypes.data_as(ct.POINTER(ct.c_double))) == 0
    ref = scipy.special.jv(np.arange(n), alpha)
    np.testing.assert_allclose(out, ref, rtol=0, atol=2e-16 * max(1.0, alpha))
    big = ref != 0
    assert np.all(np.abs(out[big] - ref[big]) <= 1e-12 * np.abs(ref[big]) + 1e-300) or alpha > 20


def test_bessel_rejects_bad_args(lib):
    out = np.zeros(4)
    p = out.ctypes.data_as(ct.POINTER(ct.c_double))
    assert lib.kt_bessel_j(-1.0, 4, p) == -1
    assert lib.kt_bessel_j(1.0, 0, p) == -1
    assert lib.kt_bessel_j(1.0, 257, p) == -1


def _make(net, **over):
    from paper_1801_04382_gb300 import Problem
    nt, M = 10, 4
    eps = si.guess_pulses(net.n_ctrl, nt, 5.0, 1.0)
    kw = dict(T=5.0, nt=nt, M=M, eps_guess=eps, shape=si.shape_functions(net.n_ctrl, nt, 5.0),
              lam=np.full(net.n_ctrl, 10.0), uniforms=si.uniforms(0, 2, M, 5))
    kw.update(over)
    return Problem(net, **kw)


def test_validation_errors_before_device_calls(lib):
    from paper_1801_04382_gb300 import KrotovError
    net = pm.cascaded_chain(2, 1)
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        _make(net, nt=0)
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        _make(net, lam=np.array([10.0, -1.0]))
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        _make(net, uniforms=si.uniforms(0, 2, 4, 4))        # even draws_per_traj
    bad = pm.cascaded_chain(2, 1)
    bad.ctrl_node = np.array([0, 5], dtype=np.int32)
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        _make(bad)
    bad = pm.cascaded_chain(2, 1)
    bad.a_local = bad.a_local + np.eye(bad.n_loc)            # two entries per row: not a ladder factor
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        _make(bad)
    eps = si.guess_pulses(2, 10, 5.0, 1.0)
    eps[0, 3] = np.nan
    with pytest.raises(KrotovError, match="KT_ERR_NONFINITE"):
        _make(net, eps_guess=eps)
    with pytest.raises(KrotovError, match="KT_ERR_RANGE"):
        _make(net, eps_bound=0.5)
    with pytest.raises(KrotovError, match="KT_ERR_UNSUPPORTED"):
        _make(pm.cascaded_chain(9, 1))
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        _make(net, tile_traj=-2)


def test_batch_validation_before_device_calls(lib):
    from paper_1801_04382_gb300 import Batch, KrotovError
    with pytest.raises(KrotovError, match="KT_ERR_ARG"):
        Batch([])
    net = pm.cascaded_chain(2, 1)
    nt, M = 10, 4
    spec = dict(net=net, T=5.0, nt=nt, M=M, eps_guess=si.guess_pulses(2, nt, 5.0, 1.0),
                shape=si.shape_functions(2, nt, 5.0), lam=np.full(2, 10.0), uniforms=si.uniforms(0, 2, M, 5))
    with pytest.raises(KrotovError, match="problem 0: .*lambda"):
        Batch([dict(spec, lam=np.array([10.0, 0.0])), spec])


def test_model_builder_matches_paper_structure():
    """Product-side model factors: Hermitian node and control factors, ladder factor with one
    entry per row/column, Hermitian cascade pair list (Eq. ham_interaction), and sqrt(2 kappa)
    Lindblad coefficients (Sec. 3.1)."""
    net = pm.cascaded_chain(3, 2, kappa=0.7)
    for h in list(net.h0_local) + list(net.hc_local):
        assert np.abs(h - h.conj().T).max() == 0.0
    assert np.all((net.a_local != 0).sum(axis=0) <= 1) and np.all((net.a_local != 0).sum(axis=1) <= 1)
    pairs = {(int(d), int(s)): c for d, s, c in zip(net.pair_dst, net.pair_src, net.pair_coef)}
    for (d, s), c in pairs.items():
        assert pairs[(s, d)] == np.conj(c)
        if d < s:
            assert c == pytest.approx(0.7j)
    assert np.allclose(net.lind_coef, np.sqrt(1.4))
    assert abs(np.linalg.norm(net.psi_tgt) - 1.0) < 1e-15


@pytest.mark.parametrize("N,nc,kappa,g,lind", [(2, 1, 1.0, 1.0, "collective"), (2, 2, 0.7, 1.0, "collective"),
                                               (3, 1, 1.3, 1.0, "collective"), (1, 2, 1.0, 1.0, "collective"),
                                               (2, 2, 1.0, complex(0.8, 0.6), "collective"),
                                               (2, 3, 1.0, 1.0, "collective"), (3, 2, 1.0, 1.0, "local")])
def test_structured_generator_tables_match_dense_heff(lib, N, nc, kappa, g, lind):
    """The library's structured generator tables, expanded with the kernels' own indexing
    (digits, slot offsets, per-direction pair tables), equal the oracle's dense
    H_eff = H - (i/2) L^dag L (direction 0) and -H_eff^dag (direction 1, co-state propagation).
    Includes a complex cavity coupling (tables of the complex cavity-structure path) and cavity
    cutoff 3 (tables of the strided path), and one Lindblad operator per node (no L^dag L cross
    terms: the cascade keeps both hop directions)."""
    from oracle import model as om
    from paper_1801_04382_gb300.problem import generator_dense
    net = pm.cascaded_chain(N, nc, kappa=kappa, g=g, lindblad=lind)
    m = om.build_model(N, nc, kappa=kappa, g=g, lindblad=lind)
    nt, T, M = 8, 1.0, 3
    rng = np.random.default_rng(N * 10 + nc)
    eps_guess = si.guess_pulses(N, nt, T, 2.0)
    args = (net, T, nt, M, eps_guess, si.shape_functions(N, nt, T), np.full(N, 10.0), si.uniforms(0, 1, M, 5))
    for trial in range(3):
        eps = rng.uniform(-2.0, 2.0, size=N)
        Heff = m.Heff(eps)
        scale = np.abs(Heff).max()
        G0 = generator_dense(*args, eps=eps, direction=0)
        G1 = generator_dense(*args, eps=eps, direction=1)
        assert np.abs(G0 - Heff).max() <= 1e-12 * scale
        assert np.abs(G1 + Heff.conj().T).max() <= 1e-12 * scale


@pytest.mark.parametrize("N,nc,lind", [(1, 1, "collective"), (1, 2, "collective"), (2, 1, "collective"),
                                       (2, 1, "local")])
def test_liouville_generator_tables_match_oracle_liouvillian(lib, N, nc, lind):
    """Density-matrix problems: the library's Liouville-space generator G (2N nodes, lower-lower pair
    hops for L rho L^dag, a ket and a bra term per control), expanded with the kernels' indexing, equals
    i times the oracle's Liouvillian of Eq. lindblad (d vec(rho)/dt = L vec(rho) = -i G vec(rho)), and
    the adjoint direction equals -G^dag (the co-state P runs under the adjoint dynamics)."""
    from oracle import lindblad as ol
    from oracle import model as om
    from paper_1801_04382_gb300.problem import generator_dense
    net = pm.cascaded_chain(N, nc, lindblad=lind)
    m = om.build_model(N, nc, lindblad=lind)
    nt, T = 8, 1.0
    args = (net, T, nt, 1, si.guess_pulses(N, nt, T, 2.0), si.shape_functions(N, nt, T), np.full(N, 10.0),
            si.uniforms(0, 1, 1, 5))
    rng = np.random.default_rng(7 + N + nc)
    for _ in range(2):
        eps = rng.uniform(-2.0, 2.0, size=N)
        G = 1j * ol.liouvillian(m.Heff(eps), m.L).toarray()
        scale = np.abs(G).max()
        G2 = generator_dense(*args, eps=eps, direction=2)
        G3 = generator_dense(*args, eps=eps, direction=3)
        assert np.abs(G2 - G).max() <= 1e-12 * scale
        assert np.abs(G3 + G.conj().T).max() <= 1e-12 * scale


@pytest.mark.parametrize("N,nc,ipts", [(2, 2, (0, 1, 4)), (3, 2, (0, 2, 4))])
def test_generator_tables_of_every_thread_mapping_match_dense_heff(lib, N, nc, ipts):
    """The tables of the automatic mapping (d = 81: the strided one-item mapping; d = 729: the
    cavity-structure fiber mapping with its real / imaginary slot order and kernel-parameter
    constants) and of the strided mapping at 1, 2 or 4 items per thread (an FP64 tile holds at most
    512 threads) all expand to the oracle's H_eff and -H_eff^dag."""
    from oracle import model as om
    from paper_1801_04382_gb300.problem import generator_dense
    net = pm.cascaded_chain(N, nc)
    m = om.build_model(N, nc)
    nt, T, M = 8, 1.0, 3
    args = (net, T, nt, M, si.guess_pulses(N, nt, T, 2.0), si.shape_functions(N, nt, T), np.full(N, 10.0),
            si.uniforms(0, 1, M, 5))
    eps = np.random.default_rng(N).uniform(-2.0, 2.0, size=N)
    Heff = m.Heff(eps)
    Heff = Heff.toarray() if hasattr(Heff, "toarray") else Heff
    scale = np.abs(Heff).max()
    for ipt in ipts:
        G0 = generator_dense(*args, eps=eps, direction=0, items_per_thread=ipt)
        G1 = generator_dense(*args, eps=eps, direction=1, items_per_thread=ipt)
        assert np.abs(G0 - Heff).max() <= 1e-12 * scale, ipt
        assert np.abs(G1 + Heff.conj().T).max() <= 1e-12 * scale, ipt


def test_items_per_thread_must_be_a_power_of_two_up_to_16(lib):
    from paper_1801_04382_gb300.problem import generator_dense
    net = pm.cascaded_chain(2, 1)
    nt, T, M = 8, 1.0, 3
    args = (net, T, nt, M, si.guess_pulses(2, nt, T, 2.0), si.shape_functions(2, nt, T), np.full(2, 10.0),
            si.uniforms(0, 1, M, 5))
    for bad in (3, 32, -2):
        with pytest.raises(Exception, match="items_per_thread"):
            generator_dense(*args, eps=np.zeros(2), direction=0, items_per_thread=bad)
