"""Whole-sweep launches (kt_config.per_interval_launches = 0, the default): a problem whose tiles are
all resident at once and which keeps every co-state runs each sweep as one launch -- the backward
sweep a plain one, the forward sweep a cooperative one whose CTAs meet at a grid barrier after each
interval to form the next interval's update (Sec. 2.2).  The results must equal those of the
per-interval launches bit for bit: the same arithmetic in the same order, only the launch
boundaries differ."""
import numpy as np
import pytest

import synth_inputs as si
from paper_1801_04382_gb300 import DensityProblem, Problem, cascaded_chain

pytestmark = pytest.mark.gpu


def _case(N, nc, T, nt, M, amp, seed, random_init):
    eps = si.guess_pulses(N, nt, T, amp)
    S = si.shape_functions(N, nt, T)
    lam = np.full(N, 10.0)
    U = si.uniforms(seed, 4, M, 1 + 2 * N * (1 + nc))
    d = (3 * (nc + 1)) ** N
    psi0 = si.random_states(seed + 100, M, d) if random_init else None
    return eps, S, lam, U, psi0


def _run(net, T, nt, M, eps, S, lam, U, psi0, per_interval, **kw):
    out = {}
    with Problem(net, T, nt, M, eps, S, lam, U, psi0_batch=psi0, per_interval_launches=per_interval, **kw) as p:
        out["whole"] = p.info.whole_sweep
        out["F"] = [p.forward(False)]
        out["recs"] = [p.records()]
        out["psi"] = [p.states()]
        out["tau"] = [p.fidelity()[1]]
        for _ in range(2):                      # sweep by sweep
            p.backward()
            out["chi0"] = p.costate(0)
            out["F"].append(p.forward(True))
            out["recs"].append(p.records())
            out["psi"].append(p.states())
            out["tau"].append(p.fidelity()[1])
            out["deps"] = p.deps()
        JT, _ = p.update(2)                     # graph-captured iterations
        out["JT"] = np.asarray(JT)
        out["eps"] = p.pulses()
    return out


def _same(a, b):
    assert a["F"] == b["F"]
    assert a["recs"] == b["recs"]
    for x, y in zip(a["psi"], b["psi"]):
        assert np.array_equal(x, y)
    for x, y in zip(a["tau"], b["tau"]):
        assert np.array_equal(x, y)
    for k in ("chi0", "deps", "JT", "eps"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision,scheme", [("fp64", "bisection"), ("fp32", "bisection"), ("fp64", "first_order")])
def test_whole_sweep_equals_per_interval_launches_with_jumps(precision, scheme):
    """Strong drive and random initial states (several jumps per trajectory, jumps in one interval),
    ragged last tile (M = 13): guess sweep, two sweep-by-sweep iterations, two graph iterations."""
    N, nc, T, nt, M = 2, 1, 12.0, 120, 13
    eps, S, lam, U, psi0 = _case(N, nc, T, nt, M, 30.0, 9, True)
    net = cascaded_chain(N, nc)
    a = _run(net, T, nt, M, eps, S, lam, U, psi0, False, precision=precision, jump_scheme=scheme)
    b = _run(net, T, nt, M, eps, S, lam, U, psi0, True, precision=precision, jump_scheme=scheme)
    assert a["whole"] == 1 and b["whole"] == 0
    assert sum(len(r) for recs in a["recs"] for r in recs) >= 10
    _same(a, b)


def test_whole_sweep_d81_many_tiles():
    """d = 81, 128 trajectories from the paper's initial state, FP32-mixed: 128 one-trajectory tiles
    (every one resident), and 32 four-trajectory tiles with two items per thread."""
    N, nc, T, nt, M = 2, 2, 5.0, 100, 128
    eps, S, lam, U, _ = _case(N, nc, T, nt, M, 30.0, 1, False)
    net = cascaded_chain(N, nc)
    for kw in ({}, {"tile_traj": 4, "items_per_thread": 2}):
        a = _run(net, T, nt, M, eps, S, lam, U, None, False, precision="fp32", **kw)
        b = _run(net, T, nt, M, eps, S, lam, U, None, True, precision="fp32", **kw)
        assert a["whole"] == 1
        _same(a, b)


def test_whole_sweep_density_matrix():
    """A density matrix (one Liouville-space state, one tile): two Krotov iterations."""
    N, nc, T, nt = 1, 2, 4.0, 200
    net = cascaded_chain(N, nc)
    eps = si.guess_pulses(N, nt, T, 1.0)
    S = si.shape_functions(N, nt, T)
    lam = np.full(N, 10.0)
    res = []
    for per_interval in (False, True):
        with DensityProblem(net, T, nt, eps, S, lam, per_interval_launches=per_interval) as p:
            assert p.info.whole_sweep == (0 if per_interval else 1)
            p.forward(False)
            JT, _ = p.update(2)
            res.append((np.asarray(JT), p.pulses(), p.rho()))
    for x, y in zip(res[0], res[1]):
        assert np.array_equal(x, y)


def test_large_problems_and_checkpoints_keep_per_interval_launches():
    """Whole sweeps need the strided mapping, every tile resident and every co-state kept: co-state
    checkpoints, 4096 one-trajectory tiles of d = 729, or the fiber mapping keep one launch per
    interval."""
    N, nc, T, nt = 2, 1, 1.0, 10
    eps, S, lam, U, _ = _case(N, nc, T, nt, 13, 1.0, 3, False)
    with Problem(cascaded_chain(N, nc), T, nt, 13, eps, S, lam, U, ckpt_interval=3) as p:
        assert p.info.whole_sweep == 0
    N, nc, M = 3, 2, 4096
    eps, S, lam, U, _ = _case(N, nc, T, nt, M, 1.0, 3, False)
    with Problem(cascaded_chain(N, nc), T, nt, M, eps, S, lam, U, precision="fp32", tile_traj=1,
                 items_per_thread=4) as p:
        assert p.info.n_tiles == M and p.info.whole_sweep == 0
    with Problem(cascaded_chain(N, nc), T, nt, 8, eps, S, lam, U[:, :8], precision="fp32") as p:
        assert p.info.items_per_thread == 0 and p.info.whole_sweep == 0
