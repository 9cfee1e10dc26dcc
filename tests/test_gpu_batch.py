"""Graph-captured Krotov iterations, batches of independent problems and the tile autotuner,
checked through the C ABI.

- krotov_update (one graph launch per iteration) gives bit-identical pulses, records and J_T to
  the same iterations issued sweep by sweep (propagate_backward / propagate_forward(update=1)),
  with and without co-state checkpointing.
- krotov_set_uniforms restarts the device-side pass counter at row 0.
- A batch of problems of different sizes, precisions and decay rates (the trajectories of one
  problem are independent of every other problem, Sec. 2.3) gives, problem by problem, results
  bit-identical to each problem optimised alone.
- An autotuned tile width is one of the compiled widths and the optimisation still matches the
  FP64 oracle to 1e-10.
"""
import numpy as np
import pytest

import synth_inputs as si
from oracle import mcwf
from oracle import model as om
from paper_1801_04382_gb300 import Batch, Problem, cascaded_chain

pytestmark = pytest.mark.gpu


def spec(N, nc, T, nt, M, amp, seed, n_passes, kappa=1.0, precision="fp64", ckpt=0, random_init=True, tile=0,
         update_rule="independent", jump_scheme="bisection"):
    draws = 1 + 2 * N * (1 + nc)
    d = (3 * (nc + 1)) ** N
    return dict(net=cascaded_chain(N, nc, kappa=kappa), T=T, nt=nt, M=M,
                eps_guess=si.guess_pulses(N, nt, T, amp), shape=si.shape_functions(N, nt, T),
                lam=np.full(N, 10.0), uniforms=si.uniforms(seed, n_passes, M, draws), precision=precision,
                ckpt_interval=ckpt, tile_traj=tile, update_rule=update_rule, jump_scheme=jump_scheme,
                psi0_batch=si.random_states(seed + 100, M, d) if random_init else None)


def problem(sp):
    kw = {k: sp[k] for k in ("precision", "ckpt_interval", "tile_traj", "psi0_batch", "update_rule", "jump_scheme")}
    return Problem(sp["net"], sp["T"], sp["nt"], sp["M"], sp["eps_guess"], sp["shape"], sp["lam"], sp["uniforms"],
                   **kw)


@pytest.mark.parametrize("ckpt,rule,scheme", [(0, "independent", "bisection"), (7, "independent", "bisection"),
                                              (7, "cross", "bisection"), (0, "independent", "first_order")])
def test_graph_iterations_match_sweeps(ckpt, rule, scheme):
    sp = spec(2, 1, 12.0, 120, 13, 30.0, 9, 4, ckpt=ckpt, update_rule=rule, jump_scheme=scheme)
    with problem(sp) as a, problem(sp) as b:
        a.forward(False)
        F_a, eps_a, rec_a = [], [], []
        for _ in range(3):
            a.backward()
            F_a.append(a.forward(True))
            eps_a.append(a.pulses())
            rec_a.append(a.records())
        JT, _ = b.update(1)
        JT2, _ = b.update(2)
        JT = np.concatenate([JT, JT2])
        assert np.array_equal(JT, 1.0 - np.array(F_a))
        assert np.array_equal(b.pulses(), eps_a[-1])
        assert b.records() == rec_a[-1]
        assert sum(len(r) for r in rec_a[-1]) >= 5


@pytest.mark.parametrize("where", ["host", "device"])
def test_set_uniforms_restarts_pass_counter(where):
    """krotov_set_uniforms takes host or device memory (a CUDA tensor is copied device to device)."""
    sp = spec(2, 1, 12.0, 120, 13, 30.0, 9, 3)
    with problem(sp) as a, problem(sp) as b:
        a.update(2)
        if where == "device":
            import torch
            a.set_uniforms(torch.tensor(sp["uniforms"], device="cuda"))
        else:
            a.set_uniforms(sp["uniforms"])
        b.set_pulses(a.pulses())
        assert a.forward(False) == b.forward(False)
        assert a.records() == b.records()


def mixed_specs():
    return [spec(2, 1, 12.0, 120, 13, 30.0, 9, 3, kappa=1.0),
            spec(2, 2, 5.0, 100, 40, 30.0, 3, 3, kappa=0.7, precision="fp32", ckpt=9),
            spec(3, 2, 0.5, 20, 6, 30.0, 2, 3, kappa=1.6, precision="fp32"),
            spec(2, 2, 5.0, 100, 7, 30.0, 5, 3, kappa=1.9, random_init=False),
            spec(2, 1, 12.0, 120, 9, 30.0, 4, 3, kappa=1.2, update_rule="cross", jump_scheme="first_order")]


def test_batch_matches_problems_alone():
    specs = mixed_specs()
    with Batch(specs) as bt:
        JT = bt.update(2)
        assert JT.shape == (2, len(specs))
        info = bt.info()
        assert info["n_problems"] == len(specs) and info["graph_nodes"] > 0
        got = [(p.pulses(), p.records(), p.fidelity()[0]) for p in bt.problems]
    for i, sp in enumerate(specs):
        with problem(sp) as p:
            JT_i, _ = p.update(2)
            assert np.array_equal(JT[:, i], JT_i), i
            assert np.array_equal(got[i][0], p.pulses()), i
            assert got[i][1] == p.records(), i
            assert got[i][2] == p.fidelity()[0], i


def test_batch_members_stay_usable():
    specs = mixed_specs()[:2]
    with Batch(specs) as bt:
        bt.update(1)
        p0 = bt.problems[0]
        p0.backward()
        F = p0.forward(True)
        JT = bt.update(1)
        assert 0.0 <= F <= 1.0 and np.all((JT >= 0) & (JT <= 1))


def test_autotuned_tile_matches_oracle():
    sp = spec(2, 1, 12.0, 120, 13, 30.0, 9, 2, tile=-1)
    m = om.build_model(2, 1)
    res = mcwf.optimize(m, sp["eps_guess"], sp["T"], sp["uniforms"], sp["shape"], sp["lam"], 1,
                        psi0=sp["psi0_batch"], keep=True)
    with problem(sp) as p:
        assert p.info.tile_traj in (1, 2, 4, 8, 16, 32)
        JT, _ = p.update(1)
        dmax = np.abs(res.forward[1].deps).max()
        assert abs(JT[0] - res.JT[1]) <= 1e-10
        assert np.abs(p.deps() - res.forward[1].deps).max() <= 1e-10 * dmax


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_is_bit_identical(precision):
    """Optimise 3 iterations in one go, or 1 iteration, checkpoint, and resume in a new problem
    for 2 more: identical J_T, pulses and jump records."""
    sp = spec(2, 1, 12.0, 120, 13, 30.0, 9, 5, precision=precision)
    with problem(sp) as a:
        a.forward(False)
        JT_a, _ = a.update(3)
        eps_a, rec_a = a.pulses(), a.records()
    with problem(sp) as b:
        b.forward(False)
        b.update(1)
        ck = b.checkpoint()
    assert ck["passes"] == 2
    sp2 = dict(sp, eps_guess=ck["eps"], uniforms=sp["uniforms"][ck["passes"] - 1:])
    kw = {k: sp2[k] for k in ("precision", "ckpt_interval", "tile_traj", "psi0_batch", "update_rule", "jump_scheme")}
    with Problem(sp2["net"], sp2["T"], sp2["nt"], sp2["M"], sp2["eps_guess"], sp2["shape"], sp2["lam"],
                 sp2["uniforms"], eps_bound=ck["eps_bound"], **kw) as c:
        c.forward(False)
        JT_c, _ = c.update(2)
        assert np.array_equal(JT_c, JT_a[1:])
        assert np.array_equal(c.pulses(), eps_a)
        assert c.records() == rec_a
