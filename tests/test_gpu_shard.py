"""Trajectory sharding (Sec. 2.3: trajectories are independent, only the update's scalars are
exchanged): a problem split into shards gives the unsharded problem's results bit for bit.

* A group of shards in one process (krotov_group_*): the per-interval tile partials are copied
  between the shards' device buffers before every shard forms Delta eps in the single-GPU order.
* One NCCL shard (world size 1, the only size one GPU allows): the same sweep with the in-place
  all-gathers of the partials and of tau, inside krotov_update's CUDA graphs.
Compared: J_T per iteration, the pulse, every trajectory's jump record and final state.
"""
import numpy as np
import pytest

import synth_inputs as si
from paper_1801_04382_gb300 import Problem, ShardGroup, cascaded_chain, nccl_unique_id, shard_ranges
from paper_1801_04382_gb300.problem import nccl_library_path

pytestmark = pytest.mark.gpu


def _case(M=16, nt=120, seed=9):
    N, nc, T = 2, 1, 12.0
    net = cascaded_chain(N, nc)
    eps0 = si.guess_pulses(N, nt, T, 30.0)
    S = si.shape_functions(N, nt, T)
    lam = np.full(N, 10.0)
    U = si.uniforms(seed, 4, M, 1 + 2 * N * (1 + nc))
    psi0 = si.random_states(seed + 100, M, net.d)
    return net, T, nt, eps0, S, lam, U, psi0


def _full(n_iter, M=16, tile=4, ckpt=0, **kw):
    net, T, nt, eps0, S, lam, U, psi0 = _case(M)
    with Problem(net, T, nt, M, eps0, S, lam, U, psi0_batch=psi0, tile_traj=tile, ckpt_interval=ckpt, **kw) as p:
        F0 = p.forward(False)
        JT, _ = p.update(n_iter)
        return F0, JT, p.pulses(), p.records(), p.states()


@pytest.mark.parametrize("sizes,ckpts", [((8, 8), (0, 0)), ((4, 12), (7, 0))])
def test_group_of_shards_equals_the_unsharded_problem(sizes, ckpts):
    M, tile, n_iter = 16, 4, 2
    F0, JT, eps, recs, psiT = _full(n_iter, M, tile)
    net, T, nt, eps0, S, lam, U, psi0 = _case(M)
    shards, off = [], 0
    for m, ck in zip(sizes, ckpts):
        shards.append(Problem(net, T, nt, m, eps0, S, lam, U[:, off:off + m], psi0_batch=psi0[off:off + m],
                              tile_traj=tile, ckpt_interval=ck, traj_offset=off, M_total=M))
        off += m
    try:
        with ShardGroup(shards[::-1]) as g:              # any order: the group sorts by offset
            JT_g = g.update(n_iter)
            F_last = g.fidelity()
        assert np.array_equal(JT_g, JT), (JT_g, JT)
        assert 1.0 - F_last == JT[-1]
        for p in shards:
            assert np.array_equal(p.pulses(), eps)
        assert sum((p.records() for p in shards), []) == recs
        assert np.array_equal(np.concatenate([p.states() for p in shards]), psiT)
        assert sum(len(r) for r in recs) >= 5
    finally:
        for p in shards:
            p.close()


def test_shard_outside_a_group_is_refused():
    net, T, nt, eps0, S, lam, U, psi0 = _case(16)
    with Problem(net, T, nt, 8, eps0, S, lam, U[:, :8], psi0_batch=psi0[:8], tile_traj=4, traj_offset=0,
                 M_total=16) as p:
        with pytest.raises(Exception, match="group"):
            p.forward(False)


def test_nccl_shard_of_world_size_one_equals_the_unsharded_problem():
    """krotov_update's graphs with the per-interval in-place all-gather of the tile partials and the
    end-of-sweep all-gather of tau over an NCCL communicator of one rank."""
    lib = nccl_library_path()
    try:
        uid = nccl_unique_id(lib)
    except Exception as e:                 # pragma: no cover - the GPU image ships NCCL with torch
        pytest.skip(f"NCCL not loadable: {e}")
    M, tile, n_iter = 16, 4, 2
    F0, JT, eps, recs, psiT = _full(n_iter, M, tile)
    net, T, nt, eps0, S, lam, U, psi0 = _case(M)
    (off, m), = shard_ranges(M, 1, tile)
    with Problem(net, T, nt, m, eps0, S, lam, U, psi0_batch=psi0, tile_traj=tile, traj_offset=off, M_total=M) as p:
        p.shard_nccl(uid, 0, 1, lib)
        assert p.forward(False) == F0
        JT_s, _ = p.update(n_iter)
        assert np.array_equal(JT_s, JT)
        assert np.array_equal(p.pulses(), eps)
        assert p.records() == recs
        assert np.array_equal(p.states(), psiT)
