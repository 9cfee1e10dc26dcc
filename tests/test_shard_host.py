"""Partition and ordering logic of trajectory sharding on CPU ranks (gloo, world size 2): each rank
takes its slice (shard_ranges) of the trajectories and of the seeded uniforms, and its tiles' update
partials land, after the all-gather, at the positions the unsharded problem uses -- so any summation
order over the gathered array is the single-GPU order."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import synth_inputs as si


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, M_total, tile, q):
    import torch
    import torch.distributed as dist
    from paper_1801_04382_gb300.problem import shard_ranges
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, m = shard_ranges(M_total, world, tile)[rank]
        U = si.uniforms(4, 3, M_total, 9)
        mine = torch.from_numpy(np.ascontiguousarray(U[:, off:off + m]))
        got = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(got, mine)
        # per-tile partials of this shard's tiles (a stand-in value per global tile and control), written
        # at the shard's tile offset of a global array and exchanged in place
        n_tiles = M_total // tile
        part = torch.zeros((n_tiles, 3), dtype=torch.float64)
        t0 = off // tile
        for t in range(m // tile):
            part[t0 + t] = torch.tensor([np.sin(t0 + t + 0.1 * c) for c in range(3)], dtype=torch.float64)
        slices = [torch.empty((m // tile, 3), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(slices, part[t0:t0 + m // tile].clone())
        q.put((rank, off, m, torch.cat(got, dim=1).numpy(), torch.cat(slices).numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_gather_in_trajectory_order():
    world, M_total, tile = 2, 1024, 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, M_total, tile, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    U = si.uniforms(4, 3, M_total, 9)
    ref = np.array([[np.sin(t + 0.1 * c) for c in range(3)] for t in range(M_total // tile)])
    covered = []
    for rank, off, m, U_all, part_all in out:
        assert np.array_equal(U_all, U)                 # the slices, gathered in rank order, are the full array
        assert np.array_equal(part_all, ref)            # tile t of the whole problem sits at row t
        covered.append((off, m))
    assert covered == [(0, 512), (512, 512)]


def test_shard_ranges_rejects_partial_tiles():
    import pytest
    from paper_1801_04382_gb300.problem import shard_ranges
    with pytest.raises(ValueError):
        shard_ranges(1000, 3, 1)
    with pytest.raises(ValueError):
        shard_ranges(1024, 2, 32 * 3)
    assert shard_ranges(96, 3, 32) == [(0, 32), (32, 32), (64, 32)]
