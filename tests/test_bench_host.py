"""Host logic of bench.py (CPU only): max-over-ranks timing with two gloo ranks, clock-log
parsing, and the nonzero count of H_eff used for the flop roofline."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
from paper_1801_04382_gb300 import model as pm


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 95.0][rank]
    out[rank] = bench.reduce_max(ms, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert dict(out) == {0: 120.0, 1: 120.0}
    assert bench.reduce_max(7.0, None, "cpu") == 7.0


def test_clock_log_parsing(tmp_path):
    path = tmp_path / "clk.csv"
    path.write_text("0, 1950, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1200.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                    "1, 300, 2070, 50.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1990, 2070, 1300.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n")

    class _P:
        def terminate(self): pass
        def wait(self, timeout=None): return 0

    fh = open(tmp_path / "dummy", "w")
    c = bench.clocks_stop(_P(), fh, str(path), 0)
    assert c["sm_mhz"] == 1980.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3


def test_average_row_nonzeros_of_four_node_chain():
    """d = 6561 chain: 1 (diagonal) + 4 x 10/9 node off-diagonals + 6 pairs x 4/9 = 8.11."""
    net = pm.cascaded_chain(4, 2)
    assert bench.avg_row_nonzeros(net) == pytest.approx(1 + 4 * 10 / 9 + 6 * 4 / 9)


def test_batch_mix_is_seeded_and_fits_its_memory_budget():
    """The 64-problem mix: deterministic for a seed, sizes in the stated ranges, and the co-state
    checkpointing chosen so that the batch holds at most the budget."""
    import synth_inputs as si
    a, b = si.batch_mix(seed=3), si.batch_mix(seed=3)
    assert a == b and len(a) == 64
    for w in a:
        assert w.n_nodes in (2, 3, 4) and w.n_cav == 2
        assert w.M in (128, 256, 512, 1024, 2048) and w.nt in (1000, 2000)
        assert 0.5 <= w.kappa <= 2.0 and w.precision == "fp32"
    held = sum(si.costate_bytes(w) + 4 * w.M * w.d * 8 for w in a)
    assert held <= 150e9
    assert any(w.ckpt_interval > 0 for w in a) and any(w.ckpt_interval == 0 for w in a)
    small = si.batch_mix(seed=3, hbm_budget=1e15)
    assert all(w.ckpt_interval == 0 for w in small)


def test_costate_bytes_counts_checkpoints_and_segment():
    import synth_inputs as si
    w = si.CONFIGS["cfg5_d6561"]
    state = w.M * w.d * 8
    assert si.costate_bytes(w) == (5000 // 100 + 1 + 100 + 1) * state
    assert si.costate_bytes(w.with_(ckpt_interval=0)) == 5001 * state
