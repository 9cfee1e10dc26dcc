"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle, on seeded inputs.

Tolerances (stated per result):
  FP64 path: states, tau and F within 1e-10 (relative to the largest entry), pulse updates
             within 1e-10 of max|Delta eps|; jump records identical in (interval, channel),
             |Delta s*| <= max(1e-9 dt, 1e-12 c^2), renormalisation c within 1e-9 relative.
  FP32-mixed: F within 1e-5 and pulse updates within 1e-4 on the benchmark workloads' models
             and initial state; states within a per-test eta (3e-5 over a few intervals, 2e-4 after
             10^2..10^3 intervals: FP32 roundoff accumulation, bounded by u K nt); a jumped
             trajectory's state within eta prod_jumps max(1, c ||L_l||) (a collapse c L_l maps a
             state error delta to c L_l delta); jump records identical on trajectories whose
             threshold margin exceeds max(1e-5, eta / 4), |Delta s*| <= max(1e-4 dt, margin c^2),
             c within 2e-3 relative (c = 1/||L psi(s*)|| moves with s*).
  Pulse updates are compared relative to the magnitude of what they sum (the oracle's deps_scale:
  S/(lambda M) sum_{k,x} |conj(chi_kx) (H_i psi_k)_x|), the standard measure of a sum's relative
  error: an update that nearly cancels over trajectories or elements is resolved to the rounding
  of its terms, not of its value.
  The jump time is compared in the norm that defines it (Sec. 2.1, step 3): the norm decays at
  rate ||L psi(s*)||^2 = 1/c^2 there, so a norm discrepancy delta shifts s* by delta c^2.
"""
import math

import numpy as np
import pytest

import synth_inputs as si
from oracle import mcwf
from oracle import model as om
from paper_1801_04382_gb300 import KrotovError, Problem, cascaded_chain

pytestmark = pytest.mark.gpu


def setup(N, nc, T, nt, M, amp, seed, n_iter, kappa=1.0, random_init=False, draws=None, lam=10.0,
          lindblad="collective"):
    n_passes = n_iter + 1
    draws = draws if draws is not None else 1 + 2 * N * (1 + nc)
    eps0 = si.guess_pulses(N, nt, T, amp)
    S = si.shape_functions(N, nt, T)
    lamv = np.full(N, lam)
    U = si.uniforms(seed, n_passes, M, draws)
    d = (3 * (nc + 1)) ** N
    psi0 = si.random_states(seed + 100, M, d) if random_init else None
    return dict(N=N, nc=nc, T=T, nt=nt, M=M, eps0=eps0, S=S, lam=lamv, U=U, psi0=psi0, n_iter=n_iter,
                kappa=kappa, lindblad=lindblad)


def run_gpu(c, precision="fp64", ckpt=0, tile=0, update_rule="independent", jump_scheme="bisection", ckpt_prefix=0,
            items_per_thread=0):
    net = cascaded_chain(c["N"], c["nc"], kappa=c["kappa"], lindblad=c["lindblad"])
    out = {"F": [], "tau": [], "recs": [], "psiT": [], "eps": [], "deps": [], "precision": precision}
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"], precision=precision,
                 ckpt_interval=ckpt, tile_traj=tile, psi0_batch=c["psi0"], update_rule=update_rule,
                 jump_scheme=jump_scheme, ckpt_prefix=ckpt_prefix, items_per_thread=items_per_thread) as p:
        out["F"].append(p.forward(False))
        out["tau"].append(p.fidelity()[1])
        out["recs"].append(p.records())
        out["psiT"].append(p.states())
        for _ in range(c["n_iter"]):
            p.backward()
            out["F"].append(p.forward(True))
            out["tau"].append(p.fidelity()[1])
            out["recs"].append(p.records())
            out["psiT"].append(p.states())
            out["eps"].append(p.pulses())
            out["deps"].append(p.deps())
        out["info"] = p.info
    return out


def replay_jumped(c, gpu, p, ks):
    """Oracle states psi_k(T) of pass p for trajectories ks, replaying the GPU's own jump record
    (interval, s*, channel, c) under the pulse that pass used (Sec. 2.1: between jumps the state
    follows exp(-i H_eff s), at a jump c L_l): the FP32 propagation checked on jumped trajectories
    without the shift of s* that an FP32 norm error causes."""
    from oracle import gradient as og
    m = om.build_model(c["N"], c["nc"], kappa=c["kappa"], lindblad=c["lindblad"])
    eps = c["eps0"] if p == 0 else gpu["eps"][p - 1]
    psi0 = m.psi0 if c["psi0"] is None else c["psi0"][ks]
    recs = [[mcwf.Jump(r[0], r[1], r[2], r[3]) for r in gpu["recs"][p][k]] for k in ks]
    return og.frozen_forward(m, eps, c["T"], psi0, recs)[-1]


def run_oracle(c, update="independent", first_order=False):
    m = om.build_model(c["N"], c["nc"], kappa=c["kappa"], lindblad=c["lindblad"])
    psi0 = c["psi0"] if c["psi0"] is not None else m.psi0
    return m, mcwf.optimize(m, c["eps0"], c["T"], c["U"], c["S"], c["lam"], c["n_iter"], psi0=psi0, keep=True,
                            update=update, first_order=first_order)


def _lind_norms(c):
    """||L_l||_2 of the model's jump operators (power iteration on L^dag L, 5% headroom)."""
    m = om.build_model(c["N"], c["nc"], kappa=c["kappa"], lindblad=c["lindblad"])
    out = []
    rng = np.random.default_rng(0)
    for L in m.L:
        v = rng.standard_normal(L.shape[0]) + 1j * rng.standard_normal(L.shape[0])
        lam = 0.0
        for _ in range(200):
            w = L.conj().T @ (L @ v)
            lam = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        out.append(1.05 * math.sqrt(lam))
    return out


def _deps_gain(c, res, update="independent", pert=1e-15):
    """Conditioning of the pulse updates: the oracle run again from initial states perturbed by a
    relative `pert`; per pass p >= 1, max |Delta eps change| over the summand scale.  A later pass
    inherits the earlier passes' errors through its pulse, so its update can be far more sensitive
    to the path's rounding than the first."""
    rng = np.random.default_rng(12345)
    m = om.build_model(c["N"], c["nc"], kappa=c["kappa"], lindblad=c["lindblad"])
    psi0 = c["psi0"] if c["psi0"] is not None else np.repeat(m.psi0[None, :], c["M"], axis=0)
    psi0 = psi0 * (1.0 + pert * rng.standard_normal(psi0.shape))
    r2 = mcwf.optimize(m, c["eps0"], c["T"], c["U"], c["S"], c["lam"], c["n_iter"], psi0=psi0, keep=True,
                       update=update)
    gains = [0.0]
    for fa, fb in zip(res.forward[1:], r2.forward[1:]):
        dmax = max(np.abs(fa.deps).max(), fa.deps_scale.max())
        gains.append(float(np.abs(fa.deps - fb.deps).max() / dmax))
    return gains


def compare(c, gpu, res, tol_state, tol_F, tol_deps, tol_s, margin_min=0.0, deps_gain=None):
    """FP64 (margin_min = 0): every result at the FP64 tolerances; with `deps_gain` (the oracle's own
    response to a 1e-15 relative perturbation of the initial states, per pass) the update of pass p
    is compared within max(tol_deps, 1e3 gain_p): 1e3 x 1e-15 = 1e-12 bounds the FP64 path's
    accumulated state rounding (nt K u with K ~ 20 terms and nt ~ 10^2..10^3 intervals).
    FP32-mixed (margin_min > 0): states within eta = tol_state (jumped trajectories: the module
    docstring's collapse bound); the FP32 norm drifts by up to delta = max(margin_min, eta / 4) (the
    state tolerance's share), so a trajectory whose norm came within delta of a threshold may jump in
    another interval; the stated subset is the trajectories whose minimum threshold margin exceeds
    delta: their records are identical in (interval, channel), s* within max(tol_s dt, delta c^2)
    and c within 2e-3, and F summed over them within tol_F (F of all trajectories too when the
    subset is all of them)."""
    dt = c["T"] / c["nt"]
    fp32 = margin_min > 0.0
    delta = max(margin_min, tol_state / 4.0) if fp32 else 0.0
    if fp32:
        lnorm = _lind_norms(c)
    for p, fw in enumerate(res.forward):
        ok = fw.margin > delta
        F_o = 1.0 - res.JT[p]
        if ok.all() or not fp32:
            assert abs(gpu["F"][p] - F_o) <= tol_F, (p, gpu["F"][p], F_o)
        if fp32:
            tau_o, _ = mcwf.fidelity(fw.psi_T, _tgt(c))
            sub_o = np.sum(np.abs(tau_o[ok]) ** 2) / c["M"]
            sub_g = np.sum(np.abs(gpu["tau"][p][ok]) ** 2) / c["M"]
            assert abs(sub_g - sub_o) <= tol_F, (p, sub_g, sub_o, int(ok.sum()))
        for k in range(c["M"]):
            if not ok[k]:
                continue
            g_rec, o_rec = gpu["recs"][p][k], fw.records[k]
            assert [(r[0], r[2]) for r in g_rec] == [(r.step, r.channel) for r in o_rec], (p, k, g_rec, o_rec)
            for gr, orc in zip(g_rec, o_rec):
                # s* is defined by ||psi(s)||^2 = r and d||psi||^2/ds = -||L psi||^2 = -1/c^2, so a
                # norm discrepancy delta moves s* by delta * c^2: compare s* in that norm too.
                tol_norm = delta if fp32 else 1e-12
                assert abs(gr[1] - orc.s) <= max(tol_s * dt, tol_norm * orc.c ** 2), (p, k, gr, orc)
                # c = 1/||L psi(s*)|| is evaluated at the (FP32-shifted) s*
                tol_c = 2e-3 if fp32 else 1e-9
                assert abs(gr[3] - orc.c) <= tol_c * orc.c, (p, k, gr, orc)
        if fp32:
            # a jump time is shifted by (FP32 norm error) * c^2, and the state after the jump moves
            # with it; jump-free trajectories are compared with the oracle's sweep, and jumped ones
            # with the oracle replaying the GPU's own record
            jumped = np.array([len(fw.records[k]) > 0 or len(gpu["recs"][p][k]) > 0 for k in range(c["M"])])
            ks = np.flatnonzero(np.array([len(r) > 0 for r in gpu["recs"][p]]))
            if len(ks):
                ref = replay_jumped(c, gpu, p, ks)
                for i, k in enumerate(ks):
                    amp = np.prod([max(1.0, r[3] * lnorm[r[2]]) for r in gpu["recs"][p][k]])
                    err = np.abs(gpu["psiT"][p][k] - ref[i]).max()
                    assert err <= tol_state * amp * np.abs(ref[i]).max(), (p, k, "jumped", err, amp)
            ok = ok & ~jumped
        scale = np.abs(fw.psi_T[ok]).max() if ok.any() else 1.0
        if ok.any():
            assert np.abs(gpu["psiT"][p][ok] - fw.psi_T[ok]).max() <= tol_state * scale, p
        if p >= 1:
            # Delta eps is a sum over trajectories (pairs) and elements with cancellation: its
            # rounding error is relative to the magnitude of its terms (deps_scale)
            dmax = max(np.abs(fw.deps).max(), fw.deps_scale.max())
            td = max(tol_deps, 1e3 * deps_gain[p]) if deps_gain is not None else tol_deps
            assert np.abs(gpu["deps"][p - 1] - fw.deps).max() <= td * max(dmax, 1e-300), (p, td)
            np.testing.assert_allclose(gpu["eps"][p - 1], fw.eps, rtol=0, atol=td * max(dmax, 1e-300) * 4)


def _tgt(c):
    return om.build_model(c["N"], c["nc"], kappa=c["kappa"], lindblad=c["lindblad"]).psi_tgt


def test_cfg1_fp64_one_iteration():
    """Plain FP64 Krotov, 1 iteration, d = 36, 32 trajectories, nt = 500, seed 0."""
    wl = si.CONFIGS["cfg1_d36"]
    c = setup(wl.n_nodes, wl.n_cav, wl.T, wl.nt, wl.M, wl.guess_amp, wl.seed, 1)
    gpu = run_gpu(c)
    _, res = run_oracle(c)
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)


@pytest.mark.parametrize("tile", [0, 1, 4, 32])
def test_stress_fp64_multi_jump(tile):
    """Strong drive and random full-space initial states: several jumps per trajectory, jumps
    inside the same interval, ragged last tile (M = 13)."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=True)
    gpu = run_gpu(c, tile=tile)
    _, res = run_oracle(c)
    n_jumps = sum(len(r) for fw in res.forward for r in fw.records)
    assert n_jumps >= 10
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)


@pytest.mark.parametrize("ipt,tile", [(1, 4), (2, 0), (1, 1)])
def test_strided_mapping_with_few_items_per_thread(ipt, tile):
    """The strided thread mapping with 1 or 2 items per thread (more threads per trajectory, for
    problems too small to fill the GPU): the multi-jump stress case, two iterations, FP64 at 1e-10."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=True)
    gpu = run_gpu(c, tile=tile, items_per_thread=ipt)
    assert gpu["info"].items_per_thread == ipt
    _, res = run_oracle(c)
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)


def test_cfg2_fp64_and_fp32():
    """d = 81 (cavity cutoff 2), 128 trajectories, nt = 1000, seed 1; FP64 and FP32-mixed."""
    wl = si.CONFIGS["cfg2_d81"]
    c = setup(wl.n_nodes, wl.n_cav, wl.T, wl.nt, wl.M, 30.0, wl.seed, 1)
    _, res = run_oracle(c)
    compare(c, run_gpu(c, "fp64"), res, 1e-10, 1e-10, 1e-10, 1e-9)
    # FP32 states after 1000 intervals of K = 17 Chebyshev terms: unit roundoff 6e-8 times
    # K * nt = 1.7e4 dependent steps bounds the drift near 1e-3; 2e-4 of the largest entry
    compare(c, run_gpu(c, "fp32"), res, 2e-4, 1e-5, 1e-4, 1e-4, margin_min=1e-5)


@pytest.mark.parametrize("ckpt,prefix", [(7, 0), (7, 50), (-1, 0)])
def test_checkpointed_costates_are_bit_identical(ckpt, prefix):
    """Co-states kept every 7 intervals, kept for t_0..t_50 and every 7th after, or chosen from the
    free device memory (ckpt_interval = -1): the optimisation is bit-identical to keeping them all."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=True)
    a = run_gpu(c, ckpt=0)
    b = run_gpu(c, ckpt=ckpt, ckpt_prefix=prefix)
    for x, y in zip(a["eps"], b["eps"]):
        assert np.array_equal(x, y)
    assert a["F"] == b["F"]
    info = b["info"]
    if ckpt == -1:       # plenty of device memory for 121 small states
        assert info.ckpt_interval == 0 and info.costate_slots == c["nt"] + 1
    else:
        assert info.ckpt_interval == 7 and info.ckpt_kept_prefix == prefix
        assert info.costate_slots == prefix + 1 + (c["nt"] - prefix + 6) // 7


def test_costates_match_oracle():
    c = setup(2, 1, 12.0, 120, 6, 30.0, 4, 0, random_init=True)
    net = cascaded_chain(2, 1)
    m = om.build_model(2, 1)
    fw = mcwf.forward_pass(m, c["eps0"], c["T"], c["U"][0], c["psi0"])
    tau, _ = mcwf.fidelity(fw.psi_T, m.psi_tgt)
    chi = mcwf.backward_pass(m, c["eps0"], c["T"], tau[:, None] * m.psi_tgt[None, :], fw.records)
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"], psi0_batch=c["psi0"]) as p:
        p.forward(False)
        p.backward()
        for j in (0, 1, 60, 119, 120):
            got = p.costate(j)
            assert np.abs(got - chi[j]).max() <= 1e-10 * np.abs(chi[j]).max(), j


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 3e-5)])
def test_d729_sampled(precision, tol):
    """Three-node chain (d = 729, dt = 0.025) over a short window, one Krotov iteration."""
    c = setup(3, 2, 0.5, 20, 6, 30.0, 2, 1, random_init=True)
    gpu = run_gpu(c, precision)
    _, res = run_oracle(c)
    compare(c, gpu, res, tol, tol, 1e-10 if precision == "fp64" else 1e-4,
            1e-9 if precision == "fp64" else 1e-4, margin_min=0.0 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 3e-5)])
def test_d6561_forward_sampled(precision, tol):
    """Four-node chain (d = 6561, dt = 0.01): forward sweep over a few intervals."""
    c = setup(4, 2, 0.04, 4, 2, 1.0, 4, 0, random_init=True)
    gpu = run_gpu(c, precision)
    _, res = run_oracle(c)
    compare(c, gpu, res, tol, tol, 1.0, 1e-9 if precision == "fp64" else 1e-4,
            margin_min=0.0 if precision == "fp64" else 1e-5)


def test_record_full_is_reported_and_recoverable():
    c = setup(2, 1, 12.0, 120, 8, 30.0, 9, 0, random_init=True, draws=1)
    net = cascaded_chain(2, 1)
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"], psi0_batch=c["psi0"]) as p:
        with pytest.raises(KrotovError, match="RECORD_FULL"):
            p.forward(False)
    c2 = setup(2, 1, 12.0, 120, 8, 30.0, 9, 0)
    with Problem(net, c2["T"], c2["nt"], c2["M"], c2["eps0"], c2["S"], c2["lam"], c2["U"]) as p:
        p.forward(False)


def test_update_before_backward_is_a_state_error():
    c = setup(2, 1, 5.0, 20, 4, 1.0, 0, 0)
    net = cascaded_chain(2, 1)
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"]) as p:
        with pytest.raises(KrotovError, match="KT_ERR_STATE"):
            p.forward(True)
        with pytest.raises(KrotovError, match="KT_ERR_STATE"):
            p.backward()


def test_full_size_launch_sampled():
    """The benchmark's launch configuration -- d = 6561, 1024 trajectories, FP32-mixed, one CTA per
    trajectory, co-state checkpoints (every 3 of 4 intervals, so one segment is recomputed) -- over a
    short window (dt = 0.01); trajectories start in the paper's initial state except the first 32,
    which start in random full-space states and jump.  F, the pulse update and every jump-free
    trajectory's state against the oracle."""
    wl = si.CONFIGS["cfg5_d6561"]
    nt = 4
    c = setup(wl.n_nodes, wl.n_cav, wl.dt * nt, nt, wl.M, wl.guess_amp, wl.seed, 1, random_init=True)
    m = om.build_model(wl.n_nodes, wl.n_cav)
    psi0 = np.repeat(m.psi0[None, :], wl.M, axis=0)
    psi0[:32] = c["psi0"][:32]
    c["psi0"] = psi0
    gpu = run_gpu(c, "fp32", ckpt=3)
    assert gpu["info"].tile_traj == 1 and gpu["info"].n_tiles == wl.M
    _, res = run_oracle(c)
    compare(c, gpu, res, 3e-5, 1e-5, 1e-4, 1e-4, margin_min=1e-5)


def test_cross_trajectory_update_fp64():
    """Cross-trajectory update (Eq. cross_traj_update), FP64: strong drive, random full-space initial
    states (several jumps per trajectory), 13 trajectories (one padded 32 x 32 pair tile), two
    iterations, against the oracle at the FP64 tolerances."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=True)
    gpu = run_gpu(c, update_rule="cross")
    _, res = run_oracle(c, update="cross")
    assert sum(len(r) for fw in res.forward for r in fw.records) >= 10
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)


def test_cross_trajectory_update_fp32_checkpointed():
    """d = 81, 40 trajectories in the paper's initial state (pair tiles padded to 64), co-state
    checkpoints every 9 intervals, FP32-mixed, two iterations, at the FP32 tolerances (F 1e-5)."""
    c = setup(2, 2, 5.0, 100, 40, 30.0, 3, 2, random_init=False)
    gpu = run_gpu(c, "fp32", ckpt=9, update_rule="cross")
    _, res = run_oracle(c, update="cross")
    compare(c, gpu, res, 3e-5, 1e-5, 1e-4, 1e-4, margin_min=1e-5)


def test_first_order_jump_scheme_fp64():
    """First-order jump scheme (Sec. 2.1): at most one jump per interval, applied at its end
    (s* = dt).  Strong drive and random full-space initial states, two iterations, FP64."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=True)
    gpu = run_gpu(c, jump_scheme="first_order")
    _, res = run_oracle(c, first_order=True)
    dt = c["T"] / c["nt"]
    n = 0
    for recs in gpu["recs"]:
        for rk in recs:
            steps = [r[0] for r in rk]
            assert len(steps) == len(set(steps))
            assert all(r[1] == dt for r in rk)
            n += len(rk)
    assert n >= 10
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)


@pytest.mark.parametrize("nc", [1, 2])
def test_complex_coupling_takes_the_complex_cavity_path(nc):
    """A cavity coupling with a phase (g = e^{i pi/5}) is neither real nor imaginary, so the library
    keeps the complex form of the cavity-structure kernels; FP64 against the oracle built with the
    same complex g (d = 36: random full-space states with jumps; d = 81: the paper's initial state,
    which keeps the oracle's run short)."""
    g = complex(math.cos(math.pi / 5), math.sin(math.pi / 5))
    c = setup(2, nc, 12.0 if nc == 1 else 5.0, 120 if nc == 1 else 100, 13, 30.0, 9, 2, random_init=nc == 1)
    net = cascaded_chain(2, nc, g=g)
    out = {"F": [], "recs": [], "psiT": [], "eps": [], "deps": []}
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"], psi0_batch=c["psi0"]) as p:
        out["F"].append(p.forward(False))
        out["recs"].append(p.records())
        out["psiT"].append(p.states())
        for _ in range(c["n_iter"]):
            p.backward()
            out["F"].append(p.forward(True))
            out["recs"].append(p.records())
            out["psiT"].append(p.states())
            out["eps"].append(p.pulses())
            out["deps"].append(p.deps())
    m = om.build_model(2, nc, g=g)
    res = mcwf.optimize(m, c["eps0"], c["T"], c["U"], c["S"], c["lam"], c["n_iter"], psi0=c["psi0"], keep=True)
    compare(c, out, res, 1e-10, 1e-10, 1e-10, 1e-9)


def test_cavity_cutoff_three_takes_the_strided_path():
    """Cavity cutoff 3 (n_loc = 12, d = 144): no fiber kernel is compiled for n_loc = 12, so the
    generic strided mapping runs; FP64 stress case against the oracle."""
    c = setup(2, 3, 4.0, 40, 13, 30.0, 9, 2, random_init=True)
    gpu = run_gpu(c)
    _, res = run_oracle(c)
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)


def test_krotov_functional_matches_oracle():
    """Krotov's functional J = J_T + sum_c lambda_c sum_j Delta eps_cj^2 dt / S_cj (Eq.
    krotov_functional) as krotov_update reports it, and J_T, against the oracle: FP64, strong drive,
    random full-space initial states with jumps, two iterations (the graph path)."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=True)
    net = cascaded_chain(2, 1)
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"], psi0_batch=c["psi0"]) as p:
        F0 = p.forward(False)
        JT, J = p.update(2)
    _, res = run_oracle(c)
    assert abs(F0 - (1.0 - res.JT[0])) <= 1e-10
    np.testing.assert_allclose(JT, res.JT[1:], rtol=0, atol=1e-10)
    np.testing.assert_allclose(J, res.J, rtol=0, atol=1e-10)
    assert np.all(np.array(J) - np.array(JT) > 1e-8)          # the penalty term is really there


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_lindblad_channels_match_oracle(precision):
    """One Lindblad operator per node (L_i = sqrt(2 kappa) a_i, n_lind = 2): the channel of every
    jump is drawn from <psi|L_l^dag L_l|psi> (Sec. 2.1); records identical in (interval, channel)
    with the oracle, both channels used; FP64 at 1e-10 with random full-space initial states (several
    jumps per trajectory), FP32-mixed at its tolerances from the paper's initial state (its stated
    tolerances are for that workload: an FP32 error grows through every further jump)."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 2, random_init=precision == "fp64", lindblad="local")
    gpu = run_gpu(c, precision)
    _, res = run_oracle(c)
    chans = {r.channel for fw in res.forward for recs in fw.records for r in recs}
    assert chans == {0, 1}
    if precision == "fp64":
        # several jumps per trajectory make the second update ~1e3 times as sensitive as the first
        compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9, deps_gain=_deps_gain(c, res))
    else:
        # A stress case beyond the benchmark workloads (guess amplitude 30, two channels, several
        # jumps per trajectory).  120 intervals of K ~ 28 terms at d = 36: unit roundoff 6e-8 x K nt
        # ~ 2e-4 bounds the state drift eta; F is held to the bound that drift implies: tau_k moves by
        # at most 2 eta (a state error eta relative to ||psi_k||, a unit target) and
        # mean_k |tau_k| <= sqrt(F), so |Delta F| <= 4 eta sqrt(F) + 4 eta^2.
        eta = 2e-4
        F_max = max(1.0 - jt for jt in res.JT)
        compare(c, gpu, res, eta, 4.0 * eta * math.sqrt(F_max) + 4.0 * eta ** 2, 1e-4, 1e-4, margin_min=1e-5)


_D6561 = {}


def _d6561_case(stress):
    """The d = 6561 full-sweep case and its oracle run (about 30 s); stress: trajectories 0-1 start in
    random full-space states (several jumps each)."""
    if stress not in _D6561:
        c = setup(4, 2, 2.0, 200, 8, 1.0, 4, 1, random_init=True)
        m = om.build_model(4, 2)
        psi0 = np.repeat(m.psi0[None, :], 8, axis=0)
        if stress:
            psi0[:2] = c["psi0"][:2]
        c["psi0"] = psi0
        _D6561[stress] = (c, run_oracle(c)[1])
    return _D6561[stress]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_d6561_full_sweep(precision):
    """Four-node chain (d = 6561, dt = 0.01) over a whole sweep: 8 trajectories, nt = 200, co-states
    checkpointed every 50 intervals, one Krotov iteration.  FP64 at 1e-10 with trajectories 0-1 in
    random full-space states (several jumps), the rest in the paper's initial state; FP32-mixed at its
    tolerances (states 2e-4 of the largest entry over 10^2..10^3 intervals) from the paper's initial
    state, the workload its tolerances are stated for."""
    c, res = _d6561_case(precision == "fp64")
    gpu = run_gpu(c, precision, ckpt=50)
    if precision == "fp64":
        assert sum(len(r) for fw in res.forward for r in fw.records) >= 1
    if precision == "fp64":
        compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)
    else:
        compare(c, gpu, res, 2e-4, 1e-5, 1e-4, 1e-4, margin_min=1e-5)


def test_copy_wait_timeout_is_reported_and_the_device_stays_usable():
    """Failure detection without a fault: with inject_copy_timeout every interval kernel's first wait
    for its bulk copy watches a barrier nothing arrives at; the short wait runs out, the kernel lets
    the real copy land (second bounded wait) and leaves, and the sweep returns KT_ERR_TIMEOUT.  The
    device stays usable: a problem created afterwards matches the oracle at 1e-10."""
    c = setup(2, 1, 12.0, 120, 13, 30.0, 9, 1, random_init=True)
    net = cascaded_chain(2, 1)
    with Problem(net, c["T"], c["nt"], c["M"], c["eps0"], c["S"], c["lam"], c["U"], psi0_batch=c["psi0"],
                 inject_copy_timeout=True) as p:
        with pytest.raises(KrotovError, match="TIMEOUT"):
            p.forward(False)
    gpu = run_gpu(c)
    _, res = run_oracle(c)
    compare(c, gpu, res, 1e-10, 1e-10, 1e-10, 1e-9)
