"""GPU gradient (krotov_gradient / KrotovTrajFunction) against the oracle's exact frozen-record
gradient and central finite differences.

FP64: dJ_T/deps within 1e-10 of max |dJ_T/deps| of the oracle (the FP64 parity tolerance);
FP32-mixed: within 2e-4 of it (complex64 propagation of states and co-states).
"""
import numpy as np
import pytest

import synth_inputs as si
from oracle import gradient as og
from oracle import mcwf
from oracle import model as om
from paper_1801_04382_gb300 import Problem, cascaded_chain

pytestmark = pytest.mark.gpu


def _records_to_oracle(recs):
    return [[mcwf.Jump(step, s, ch, c) for (step, s, ch, c) in rk] for rk in recs]


def _case(N, nc, T, nt, M, amp, seed, random_init=True, kappa=1.0):
    eps = si.guess_pulses(N, nt, T, amp)
    S = si.shape_functions(N, nt, T)
    lam = np.full(N, 10.0)
    U = si.uniforms(seed, 2, M, 1 + 2 * N * (1 + nc))
    d = (3 * (nc + 1)) ** N
    psi0 = si.random_states(seed + 50, M, d) if random_init else None
    return eps, S, lam, U, psi0


@pytest.mark.parametrize("ckpt", [0, 7])
def test_gradient_fp64_matches_oracle_with_jumps(ckpt):
    N, nc, T, nt, M = 2, 1, 6.0, 60, 6
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 30.0, 5)
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, psi0_batch=psi0, ckpt_interval=ckpt) as p:
        F = p.forward(keep_for_gradient=True)
        recs = p.records()
        grad = p.gradient().cpu().numpy()
    assert sum(len(r) for r in recs) >= 2
    m = om.build_model(N, nc)
    ref, jt = og.gradient(m, eps, T, psi0, _records_to_oracle(recs))
    assert abs((1.0 - F) - jt) <= 1e-10
    assert np.abs(grad - ref).max() <= 1e-10 * np.abs(ref).max()


def test_gradient_fp32_d729_matches_oracle():
    N, nc, T, nt, M = 3, 2, 0.25, 10, 4
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 30.0, 2)
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, psi0_batch=psi0, precision="fp32") as p:
        p.forward(keep_for_gradient=True)
        recs = p.records()
        grad = p.gradient().cpu().numpy()
    m = om.build_model(N, nc)
    ref, _ = og.gradient(m, eps, T, psi0, _records_to_oracle(recs))
    assert np.abs(grad - ref).max() <= 2e-4 * np.abs(ref).max()


def test_autograd_function_matches_central_differences_at_kappa_zero():
    torch = pytest.importorskip("torch")
    from paper_1801_04382_gb300 import trajectory_functional
    N, nc, T, nt, M = 2, 1, 5.0, 50, 3
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 30.0, 8, kappa=0.0)
    net = cascaded_chain(N, nc, kappa=0.0)
    with Problem(net, T, nt, M, eps, S, lam, U, psi0_batch=psi0) as p:
        e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
        J = trajectory_functional(e, p)
        J.backward()
        g = e.grad.cpu().numpy()
        rng = np.random.default_rng(0)
        h = 1e-4
        for _ in range(20):
            i, j = int(rng.integers(N)), int(rng.integers(nt))
            ep = eps.copy(); ep[i, j] += h
            em = eps.copy(); em[i, j] -= h
            Jp = float(trajectory_functional(torch.tensor(ep, device="cuda"), p))
            Jm = float(trajectory_functional(torch.tensor(em, device="cuda"), p))
            fd = (Jp - Jm) / (2 * h)
            assert fd == pytest.approx(g[i, j], rel=1e-6, abs=1e-11)


def test_gradient_full_size_launch_fd_and_precisions():
    """The three-node gradient workload's launch size (d = 729, 1024 trajectories, one CTA per
    trajectory in the gradient kernel) over a shorter window (nt = 200, dt = 0.025) at kappa = 0 --
    no jumps, so the free-running functional is the frozen-record one: the FP64 gradient against
    central differences (h = 1e-4) at 20 random slots, and the FP32-mixed gradient against the FP64
    one within 2e-3 of max |dJ_T/deps| (complex64 states and co-states over 200 intervals)."""
    N, nc = 3, 2
    wl = si.CONFIGS["cfg3_d729"]
    nt, M = 200, wl.M
    T = wl.dt * nt
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 30.0, wl.seed, kappa=0.0)
    net = cascaded_chain(N, nc, kappa=0.0)
    grads = {}
    for prec in ("fp64", "fp32"):
        with Problem(net, T, nt, M, eps, S, lam, U, psi0_batch=psi0, precision=prec) as p:
            p.forward(keep_for_gradient=True)
            assert sum(len(r) for r in p.records()) == 0
            grads[prec] = p.gradient().cpu().numpy()
            if prec != "fp64":
                continue
            rng = np.random.default_rng(1)
            h = 1e-4
            for _ in range(20):
                i, j = int(rng.integers(N)), int(rng.integers(nt))
                ep = eps.copy()
                ep[i, j] += h
                em = eps.copy()
                em[i, j] -= h
                p.set_pulses(ep)
                Jp = 1.0 - p.forward(False)
                p.set_pulses(em)
                Jm = 1.0 - p.forward(False)
                fd = (Jp - Jm) / (2 * h)
                assert fd == pytest.approx(grads["fp64"][i, j], rel=1e-6, abs=1e-11), (i, j)
    scale = np.abs(grads["fp64"]).max()
    assert np.abs(grads["fp32"] - grads["fp64"]).max() <= 2e-3 * scale


def test_gradient_d6561_full_launch_checkpointed_replay():
    """The four-node launch size (d = 6561, 1024 trajectories, FP32-mixed) over a short window:
    the gradient with forward states kept every 2 intervals and replayed per segment equals the
    one with every state kept, within FP32 rounding (2e-4 of max |dJ_T/deps|)."""
    N, nc = 4, 2
    wl = si.CONFIGS["cfg5_d6561"]
    nt, M = 6, wl.M
    T = wl.dt * nt
    eps, S, lam, U, _ = _case(N, nc, T, nt, M, 1.0, wl.seed, random_init=False)
    grads = []
    for ckpt in (0, 2):
        with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, precision="fp32", ckpt_interval=ckpt) as p:
            p.forward(keep_for_gradient=True)
            grads.append(p.gradient().cpu().numpy())
    scale = np.abs(grads[0]).max()
    assert scale > 0 and np.all(np.isfinite(grads[1]))
    assert np.abs(grads[1] - grads[0]).max() <= 2e-4 * scale


def test_autograd_keeps_tensors_on_the_device():
    """The pulse goes in and J_T and dJ_T/deps come out as CUDA tensors: forward and backward pass
    device pointers through the C ABI on torch's current stream (no host copy of eps or of the
    gradient); the result equals the gradient of the host-driven path (set_pulses + forward +
    krotov_gradient) bit for bit, and krotov_gradient with a pulse argument equals both."""
    torch = pytest.importorskip("torch")
    from paper_1801_04382_gb300 import trajectory_functional
    N, nc, T, nt, M = 2, 1, 6.0, 60, 6
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 30.0, 5)
    U = np.repeat(U[:1], 4, axis=0)           # every pass draws the same numbers: same records
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, psi0_batch=psi0) as p:
        e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
        J = trajectory_functional(e, p)
        assert J.is_cuda and J.dim() == 0
        J.backward()
        assert e.grad.is_cuda
        g_auto = e.grad.cpu().numpy()
        p.set_pulses(eps)
        F = p.forward(keep_for_gradient=True)
        assert abs(float(J) - (1.0 - F)) <= 1e-14
        g_host = p.gradient().cpu().numpy()
        g_arg = p.gradient(eps=torch.tensor(eps, device="cuda")).cpu().numpy()
        assert sum(len(r) for r in p.records()) >= 2
    assert np.array_equal(g_auto, g_host) and np.array_equal(g_arg, g_host)


def test_autograd_rejects_a_stale_graph_node():
    """backward of a J_T whose forward sweep was followed by another one raises instead of returning
    the later sweep's gradient."""
    torch = pytest.importorskip("torch")
    from paper_1801_04382_gb300 import trajectory_functional
    N, nc, T, nt, M = 2, 1, 2.0, 20, 2
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 3.0, 5)
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, psi0_batch=psi0) as p:
        e1 = torch.tensor(eps, device="cuda", requires_grad=True)
        J1 = trajectory_functional(e1, p)
        e2 = torch.tensor(eps * 1.1, device="cuda", requires_grad=True)
        J2 = trajectory_functional(e2, p)
        with pytest.raises(RuntimeError, match="another forward sweep"):
            J1.backward()
        J2.backward()
        assert e2.grad.is_cuda


def test_device_pulse_out_of_range_is_reported():
    """A pulse handed over in device memory is checked on the device (|eps| <= eps_bound, finite)."""
    torch = pytest.importorskip("torch")
    from paper_1801_04382_gb300 import KrotovError
    N, nc, T, nt, M = 2, 1, 2.0, 20, 2
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 3.0, 5)
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, psi0_batch=psi0) as p:
        bad = torch.tensor(eps, device="cuda")
        bad[1, 3] = 1e3
        p.set_pulses_device(bad)
        with pytest.raises(KrotovError, match="RANGE"):
            p.forward(False)
        bad[1, 3] = float("nan")
        p.set_pulses_device(bad)
        with pytest.raises(KrotovError, match="NONFINITE"):
            p.forward(False)
        p.set_pulses_device(torch.tensor(eps, device="cuda"))
        p.forward(False)
