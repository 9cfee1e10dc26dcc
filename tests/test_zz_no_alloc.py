"""The allocation-free pulse-update entry point (kt_update_overlap_noalloc).

Some callers may not allocate device memory themselves (a framework that budgets every
device allocation before the run, or code running from a callback where cudaMalloc is not
allowed).  For them the library offers the per-interval update reduction with its scratch in
a fixed device array.  This test calls it through the C ABI, twice in a row, on the initial
states and the co-states chi(t_0) of a problem, and checks its Delta eps against the one the
regular updating forward sweep (propagate_forward with the update on) applied to the first
interval, within the FP64 tolerance of the parity tests (1e-10 of max |Delta eps|).
"""
import ctypes as ct

import numpy as np
import pytest

import synth_inputs as si
from paper_1801_04382_gb300 import Problem, _capi, cascaded_chain

pytestmark = pytest.mark.gpu


def test_noalloc_update_matches_forward_sweep_on_two_calls():
    torch = pytest.importorskip("torch")
    N, nc, T, nt, M = 2, 1, 12.0, 120, 13
    net = cascaded_chain(N, nc)
    eps0 = si.guess_pulses(N, nt, T, 30.0)
    S = si.shape_functions(N, nt, T)
    lam = np.full(N, 10.0)
    U = si.uniforms(9, 2, M, 1 + 2 * N * (1 + nc))
    psi0 = si.random_states(109, M, net.d)
    with Problem(net, T, nt, M, eps0, S, lam, U, psi0_batch=psi0) as p:
        p.forward(False)
        p.backward()
        chi0 = p.costate(0)
        p.forward(True)
        ref = p.deps()[:, 0]
    assert np.abs(ref).max() > 0.0

    dev = torch.device("cuda", 0)
    psi_d = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.complex128)).to(dev)
    chi_d = torch.from_numpy(np.ascontiguousarray(chi0, dtype=np.complex128)).to(dev)
    out = torch.full((N,), np.nan, dtype=torch.float64, device=dev)
    hc = np.ascontiguousarray(np.stack([net.hc_local.real, net.hc_local.imag], axis=-1), dtype=np.float64)
    cn = np.ascontiguousarray(net.ctrl_node, dtype=np.int32)
    s0 = np.ascontiguousarray(S[:, 0])
    lib = _capi.load()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    dptr = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))
    torch.cuda.synchronize()
    for _ in range(2):
        out.fill_(np.nan)
        st = lib.kt_update_overlap_noalloc(N, net.n_loc, N, cn.ctypes.data_as(ct.POINTER(ct.c_int)), dptr(hc), M,
                                           ct.c_void_p(psi_d.data_ptr()), ct.c_void_p(chi_d.data_ptr()),
                                           dptr(s0), dptr(lam), ct.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.krotov_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (got, ref)


def test_noalloc_grid_stride_swapped_controls_and_smaller_second_call():
    """M = 1500 trajectories (more than the 1024 blocks of the fixed scratch: blocks sum several
    trajectories each), controls acting on the node other than their own index, then a second call
    with M = 13 that reuses the ticket with a smaller grid.  Reference: the definition
    Delta eps_c = S_c / (lambda_c M) sum_k Im <chi_k| H_c |psi_k> with the oracle's dense control
    operator of node ctrl_node[c], on random states, within 1e-10 of max |Delta eps|."""
    torch = pytest.importorskip("torch")
    from oracle import model as om
    N, nc = 2, 1
    net = cascaded_chain(N, nc)
    m = om.build_model(N, nc)
    cn = np.array([1, 0], dtype=np.int32)                 # control 0 on node 1, control 1 on node 0
    hc = np.ascontiguousarray(np.stack([net.hc_local.real, net.hc_local.imag], axis=-1), dtype=np.float64)
    s_j = np.array([0.37, 0.81])
    lam = np.array([10.0, 3.0])
    lib = _capi.load()
    dev = torch.device("cuda", 0)
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    dptr = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))
    for M, seed in ((1500, 31), (13, 32)):
        psi = si.random_states(seed, M, net.d)
        chi = si.random_states(seed + 1000, M, net.d)
        ref = np.array([s_j[c] / (lam[c] * M) * np.sum(np.imag(np.sum(chi.conj() * (psi @ m.Hc[cn[c]].T), axis=1)))
                        for c in range(N)])
        psi_d = torch.from_numpy(np.ascontiguousarray(psi)).to(dev)
        chi_d = torch.from_numpy(np.ascontiguousarray(chi)).to(dev)
        out = torch.full((N,), np.nan, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        st = lib.kt_update_overlap_noalloc(N, net.n_loc, N, cn.ctypes.data_as(ct.POINTER(ct.c_int)), dptr(hc), M,
                                           ct.c_void_p(psi_d.data_ptr()), ct.c_void_p(chi_d.data_ptr()),
                                           dptr(s_j), dptr(lam), ct.c_void_p(out.data_ptr()), stream)
        assert st == 0, lib.krotov_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (M, got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    lib = _capi.load()
    z = np.zeros(2 * 6 * 6 * 9)
    cn = np.zeros(9, dtype=np.int32)
    st = lib.kt_update_overlap_noalloc(2, 6, 9, cn.ctypes.data_as(ct.POINTER(ct.c_int)),
                                       z.ctypes.data_as(ct.POINTER(ct.c_double)), 4, ct.c_void_p(1), ct.c_void_p(1),
                                       z.ctypes.data_as(ct.POINTER(ct.c_double)),
                                       z.ctypes.data_as(ct.POINTER(ct.c_double)), ct.c_void_p(1), None)
    assert st == -9  # KT_ERR_UNSUPPORTED
    assert b"at most 8 controls" in lib.krotov_last_error()
