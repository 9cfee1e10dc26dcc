#!/usr/bin/env python
"""Benchmark: Krotov iterations per second of the trajectory-parallel Krotov hot path on GB300.

Workload (one "step" = one Krotov iteration = backward co-state sweep + updating forward sweep,
including any co-state recompute): four-node cascaded atom-cavity chain, three-level atoms,
cavity cutoff 2 (d = 6561), 1024 trajectories, nt = 5000 intervals of dt = 0.01, four controls,
FP32-mixed precision (complex64 states, FP64 norms and sums), co-state storage chosen from the
free device memory (all 5001 co-states, 269 GB, when they fit; --ckpt K keeps every K-th and
recomputes the rest), synthetic seeded inputs (guess pulse sin^2 of amplitude 1, uniforms from
seed 4).  The timed region runs krotov_update as the product does: one CUDA graph launch per
iteration; one more iteration launched kernel by kernel gives the per-kernel split.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--ckpt K]
    python bench.py --workload profile [--precision fp32|fp64] [--profile-M M]
    python bench.py --workload mix64 [--steps K] [--warmup W]
    python bench.py --workload grad729 [--steps K] [--warmup W]
    python bench.py --workload noise
    python bench.py --workload cross

--workload mix64 times the batch of 64 independent problems of mixed size (2, 3 and 4 nodes,
d = 81 / 729 / 6561, 128..2048 trajectories, nt 1000 or 2000, kappa in [0.5, 2], FP32-mixed,
seed 3); one step is one Krotov iteration of every problem, issued as one graph launch; the
same problems iterated one after another (one graph launch each) are timed beside it.
--workload grad729 times the exact gradient dJ_T/deps (frozen jump record) on the three-node
chain (d = 729, 1024 trajectories, nt = 2000, FP32-mixed, seed 2): one step is a forward sweep
that keeps the states plus the gradient sweep.
--workload noise measures the pulse noise nu_i (Eq. noise) after 20 Krotov iterations on the
two-node chain (d = 81, nt = 1000, guess amplitude 20 so that a quarter of the trajectories jump,
FP32-mixed) for M = 8 ... 1024 trajectories, of the pulse and of the accumulated update eps - eps_guess
(free of the smoothing residual of the smooth guess), and fits nu_i ~ M^b (the paper finds b = -1/2).
--workload density times density-matrix Krotov (Eq. krotovupdate) on the two-node d = 81 model
(vec(rho) of dimension 6561 as one Liouville-space state) in FP32-mixed and FP64.
--workload profile runs a 12-interval case of the four-node interval kernels at M trajectories (a
small command for ncu captures).
--workload cross runs 20 iterations of the cross-trajectory update (Eq. cross_traj_update) and of
the independent-trajectory update on the two-node chain (d = 81, M = 128, nt = 1000, FP32-mixed)
and reports both convergence histories, iterations/s and the pair-sum kernels' time.

N > 1 (under torchrun): every rank optimises an independent problem (its own seed); there is
no data-path collective ("weak" scaling).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

# The oracle timings run on one host thread: its sparse products use one core anyway, and a BLAS
# pool on every core makes its small dense products ~30x slower.  Set before numpy loads (the GPU
# path does no host linear algebra); a caller's own setting is kept.
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth_inputs as si  # noqa: E402

METRIC = "Krotov iters/s and traj·steps/s, FP32-mixed vs FP64 path, % of HBM roofline"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of each interval kernel at
# this workload's launch size (1024 trajectories, d = 6561, FP32-mixed), from one ncu capture of the
# current kernels (`bench.py --workload profile`, full section set: an updating forward launch and a
# backward launch); None where no capture of the current kernel exists.
NCU_TRAFFIC_PER_LAUNCH = {"bwd": None, "fwd": 108225280 + 23902976}
FP32_LANES = 128              # FP32 FMA lanes per SM (Blackwell)


def sm_count() -> int:
    """Streaming multiprocessors of the current device (read from the device, not assumed)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_peak_tflops(clk_mhz: float) -> float:
    return sm_count() * FP32_LANES * 2 * clk_mhz * 1e6 / 1e12


def executed_flops_per_elem_term(nnz: float, ri: bool) -> float:
    """FP32 flops one element of one Chebyshev term executes: every off-diagonal coupling of the
    cavity network is purely real or purely imaginary, so the kernels apply it with two FMAs
    (4 flops) instead of a complex multiply-add (8); the diagonal is a complex product (6), the
    recurrence 2 T_k - T_{k-1} 4 and the running sum a complex FMA 8."""
    return (4.0 if ri else 8.0) * (nnz - 1.0) + 6.0 + 4.0 + 8.0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(rank: int = 0, precision: str = "fp32"):
    wl = si.CONFIGS["cfg5_d6561"]
    return wl.with_(seed=wl.seed + 1000 * rank, precision=precision)


def avg_row_nonzeros(net) -> float:
    """Average nonzeros per row of the structured H_eff (diagonal counted once): node-local
    off-diagonals + pair hops, averaged over uniformly distributed digits."""
    nl, N = net.n_loc, net.n_nodes
    tot = 1.0
    for i in range(N):
        pattern = np.abs(net.h0_local[i]) > 0
        for c, node in enumerate(net.ctrl_node):
            if node == i:
                pattern |= np.abs(net.hc_local[c]) > 0
        off = pattern.sum(axis=1) - np.diag(pattern)
        tot += off.mean()
    has_lower = (np.abs(net.a_local) > 0).any(axis=1)          # row x of a nonzero
    has_raise = (np.abs(net.a_local) > 0).any(axis=0)          # column x of a nonzero -> row x of a^dag
    # pair terms of H_eff: user pairs plus L^dag L cross terms, merged; the cascade leaves
    # exactly one direction per node pair (upstream hops cancel)
    n_pairs = N * (N - 1) // 2
    tot += n_pairs * has_raise.mean() * has_lower.mean()
    return float(tot)


def reduce_max(value: float, dist, device) -> float:
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
def clocks_start(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def clocks_stop(proc, fh, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    fh.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for name, val in zip(names, parts[5:9]):
            if val.lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# ------------------------------------------------------------------------------------------
def cpu_baseline(wl, budget_s: float = 20.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: one trajectory over a
    window of the nt intervals (guess sweep, backward sweep, updating sweep), extrapolated to the
    full workload as Krotov iterations/s (oracle traj.steps: 2 sweeps x M x nt per iteration)."""
    from oracle import mcwf
    from oracle import model as om
    m = om.build_model(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    M_s = 1
    nt_s = 10
    T_s = wl.dt * nt_s
    U = si.uniforms(wl.seed, 2, M_s, wl.draws_per_traj)
    eps = si.guess_pulses(wl.n_nodes, nt_s, T_s, wl.guess_amp)
    S = si.shape_functions(wl.n_nodes, nt_s, T_s)
    lam = np.full(wl.n_nodes, wl.lam)
    cores = oracle_threads()
    t0 = time.perf_counter()
    reps = 0
    while True:
        mcwf.optimize(m, eps, T_s, U, S, lam, 1, psi0=m.psi0)
        reps += 1
        if time.perf_counter() - t0 > budget_s / 2 or reps >= 50:
            break
    el = time.perf_counter() - t0
    # per rep: guess forward + backward + updating forward = 3 sweeps of M_s * nt_s traj.steps;
    # the iteration itself is 2 of them
    traj_steps = reps * 3 * M_s * nt_s
    tsps = traj_steps / el
    iters = tsps / (2.0 * wl.M * wl.nt)
    return {"value": iters, "unit": "Krotov iters/s", "cores": cores, "kind": "oracle",
            "traj_steps_per_s": tsps,
            "sample": f"{reps} x (guess+backward+updating sweep) of {M_s} trajectory x {nt_s} intervals "
                      f"(d={wl.d}, dt={wl.dt}), extrapolated to M={wl.M}, nt={wl.nt}"}


# ------------------------------------------------------------------------------------------
def precision_comparison(stream, n_iter: int = 50):
    """FP32-mixed vs plain FP64 on the d = 81 workload (two nodes, cavity cutoff 2, 128
    trajectories, nt = 1000, seed 1): Krotov iterations/s of each path over n_iter iterations
    (CUDA events) and the final fidelities, which must agree within 1e-4."""
    import torch
    from paper_1801_04382_gb300 import Problem, cascaded_chain
    wl = si.CONFIGS["cfg2_d81"]
    net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    eps0 = si.guess_pulses(net.n_ctrl, wl.nt, wl.T, wl.guess_amp)
    S = si.shape_functions(net.n_ctrl, wl.nt, wl.T)
    lam = np.full(net.n_ctrl, wl.lam)
    U = si.uniforms(wl.seed, n_iter + 1, wl.M, wl.draws_per_traj)
    out = {"workload": f"{wl.name} (d={wl.d}, M={wl.M}, nt={wl.nt}), {n_iter} iterations"}
    for prec in ("fp32", "fp64"):
        with Problem(net, wl.T, wl.nt, wl.M, eps0, S, lam, U, precision=prec, stream=stream) as p:
            p.forward(False, stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            JT, _ = p.update(n_iter, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[f"{prec}_iters_per_s"] = n_iter * 1000.0 / ms
            out[f"{prec}_final_F"] = 1.0 - float(JT[-1])
    out["final_F_abs_diff"] = abs(out["fp32_final_F"] - out["fp64_final_F"])
    out["fp32_over_fp64"] = out["fp32_iters_per_s"] / out["fp64_iters_per_s"]
    return out


def run_mix(args, rank, world):
    """Batch of independent mixed-size problems, one graph launch per Krotov iteration."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1801_04382_gb300 import Batch, cascaded_chain

    mix = si.batch_mix(seed=3 + 1000 * rank)
    n_passes = 2 + args.warmup + args.steps
    specs, flops_it, bytes_it, tsteps_it = [], 0.0, 0.0, 0.0
    for w in mix:
        net = cascaded_chain(w.n_nodes, w.n_cav, w.delta, w.g, w.kappa)
        specs.append(dict(net=net, T=w.T, nt=w.nt, M=w.M, eps_guess=si.guess_pulses(net.n_ctrl, w.nt, w.T, w.guess_amp),
                          shape=si.shape_functions(net.n_ctrl, w.nt, w.T), lam=np.full(net.n_ctrl, w.lam),
                          uniforms=si.uniforms(w.seed, n_passes, w.M, w.draws_per_traj), precision=w.precision,
                          ckpt_interval=w.ckpt_interval, tile_traj=-1))
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    bt = Batch(specs, stream=stream)
    init_s = time.perf_counter() - t0
    for w, sp, p in zip(mix, specs, bt.problems):
        K = p.info.cheb_terms
        nnz = avg_row_nonzeros(sp["net"])
        flops_it += 2 * (8.0 * nnz + 12.0) * K * w.d * w.M * w.nt      # forward + backward sweep
        bytes_it += 5.0 * 8 * w.d * w.M * w.nt
        tsteps_it += 2.0 * w.M * w.nt
    t0 = time.perf_counter()
    bt.update(1, stream=stream)            # guess sweeps, graph capture and one iteration
    first_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        bt.update(1, stream=stream)

    clk_path = os.path.join(tempfile.gettempdir(), f"kt_clocks_{os.getpid()}.csv")
    proc, fh = clocks_start(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    JT = bt.update(args.steps, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_step = reduce_max(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    clocks = clocks_stop(proc, fh, clk_path, local)
    info = bt.info()

    # the same problems, one after another (each one graph launch per iteration)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for p in bt.problems:                  # capture each problem's own graph outside the timing
        p.update(1, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for p in bt.problems:
        p.update(1, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)

    peaks, peak_src = measured_peaks()
    clk_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = fp32_peak_tflops(clk_max)
    iters_per_s = world * 1000.0 / ms_step
    achieved = flops_it / (ms_step / 1000.0) / 1e12
    counts = {}
    for w in mix:
        counts[w.d] = counts.get(w.d, 0) + 1
    line = {
        "metric": METRIC, "value": iters_per_s, "unit": "batch Krotov iters/s (64 problems each)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": {"workload": "mix64: 64 independent problems, seed 3", "problems_by_d": counts,
                   "trajectories": sum(w.M for w in mix), "checkpointed": sum(1 for w in mix if w.ckpt_interval),
                   "tiles": "autotuned per problem", "device_bytes": info["device_bytes"],
                   "graph_kernel_nodes": info["graph_nodes"],
                   "l2": "inputs larger than L2 (co-states of all problems)", "parallelism": f"replicas{world}"},
        "traj_steps_per_s": tsteps_it * iters_per_s,
        "roofline": {"bound": "alu", "kernel": "all interval kernels of the batch", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "peak_source": f"FP32 FFMA: {sm_count()} SMs x {FP32_LANES} lanes x 2 x {clk_max:.0f} MHz"},
        "hbm_roofline": {"achieved_gbs": bytes_it * iters_per_s / world / 1e9, "peak_gbs": peaks["hbm_gbs"],
                         "frac": bytes_it * iters_per_s / world / 1e9 / peaks["hbm_gbs"], "peak_source": peak_src},
        "sequential_same_problems": {"ms_per_step": seq_ms, "batch_speedup": seq_ms / ms_step},
        "init_s": init_s, "first_iteration_s": first_s,
        "mean_final_JT": float(np.mean(JT[-1])),
        "gpu_launches": int(info["graph_nodes"]) * args.steps,
        "clocks": clocks,
    }
    bt.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_grad(args, rank, world):
    """Gradient evaluations per second on the three-node workload."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1801_04382_gb300 import Problem, cascaded_chain
    wl = si.CONFIGS["cfg3_d729"]
    wl = wl.with_(seed=wl.seed + 1000 * rank)
    net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    eps0 = si.guess_pulses(net.n_ctrl, wl.nt, wl.T, wl.guess_amp)
    S = si.shape_functions(net.n_ctrl, wl.nt, wl.T)
    lam = np.full(net.n_ctrl, wl.lam)
    U = si.uniforms(wl.seed, 1 + args.warmup + args.steps, wl.M, wl.draws_per_traj)
    stream = torch.cuda.current_stream()
    prob = Problem(net, wl.T, wl.nt, wl.M, eps0, S, lam, U, precision=wl.precision,
                   ckpt_interval=wl.ckpt_interval, stream=stream)
    info = prob.info
    for _ in range(args.warmup):
        prob.forward(False, stream=stream, keep_for_gradient=True)
        prob.gradient(stream=stream)
    clk_path = os.path.join(tempfile.gettempdir(), f"kt_clocks_{os.getpid()}.csv")
    proc, fh = clocks_start(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    prob.set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        prob.forward(False, stream=stream, keep_for_gradient=True)
        grad = prob.gradient(stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_step = reduce_max(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    prof = prob.profile()
    prob.set_profiling(False)
    clocks = clocks_stop(proc, fh, clk_path, local)
    peaks, peak_src = measured_peaks()
    clk_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = fp32_peak_tflops(clk_max)
    K = info.cheb_terms
    nnz = avg_row_nonzeros(net)
    # per control a 2d-dimensional propagation: the state's and the derivative's recurrences, plus
    # the control factor (one entry per row) applied to the state in every term
    g_ms, g_n = prof["grad"]
    flops_grad = net.n_ctrl * K * (2 * (8.0 * nnz + 12.0) + 8.0) * wl.d * wl.M
    achieved = flops_grad / (g_ms / max(g_n, 1) / 1000.0) / 1e12
    per_s = world * 1000.0 / ms_step
    line = {
        "metric": METRIC, "value": per_s, "unit": "gradient evaluations/s (forward sweep + gradient sweep)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": {"workload": "cfg3_d729 gradient", "d": wl.d, "M": wl.M, "nt": wl.nt, "dt": wl.dt,
                   "precision": "FP32-mixed", "ckpt_interval": wl.ckpt_interval, "cheb_terms": K,
                   "tile_traj": info.tile_traj, "l2": "inputs larger than L2 (forward states kept for the "
                   f"gradient, {info.device_bytes / 1e9:.1f} GB)", "parallelism": f"replicas{world}"},
        "traj_steps_per_s": per_s * 2 * wl.M * wl.nt,
        "roofline": {"bound": "alu", "kernel": "grad_kernel", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "avg_launch_ms": g_ms / max(g_n, 1), "launches": g_n, "flops_per_launch": flops_grad,
                     "peak_source": f"FP32 FFMA: {sm_count()} SMs x {FP32_LANES} lanes x 2 x {clk_max:.0f} MHz"},
        "kernels": {f"{k}_kernel": {"launches": n, "total_ms": ms, "avg_ms": ms / max(n, 1)}
                    for k, (ms, n) in prof.items() if n > 0},
        "max_abs_gradient": float(grad.abs().max()),
        "gpu_launches": int(sum(n for _, n in prof.values())),
        "clocks": clocks,
    }
    prob.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_noise(args, rank, world):
    """Pulse noise nu_i versus the number of trajectories (Fig. 4 experiment, independent trajectories)."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    if rank != 0:
        return 0
    from paper_1801_04382_gb300 import Problem, cascaded_chain
    wl = si.CONFIGS["cfg2_d81"]
    amp, n_iter = 20.0, 20
    net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    eps0 = si.guess_pulses(net.n_ctrl, wl.nt, wl.T, amp)
    S = si.shape_functions(net.n_ctrl, wl.nt, wl.T)
    lam = np.full(net.n_ctrl, wl.lam)
    stream = torch.cuda.current_stream()
    Ms = [8, 16, 32, 64, 128, 256, 512, 1024]
    rows = []
    for M in Ms:
        U = si.uniforms(wl.seed, n_iter + 1, M, wl.draws_per_traj)
        with Problem(net, wl.T, wl.nt, M, eps0, S, lam, U, precision="fp32", stream=stream) as p:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p.forward(False, stream=stream)
            e0.record(stream)
            JT, _ = p.update(n_iter, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            nu = p.pulse_noise(stream=stream)
            nu_upd = p.pulse_noise(ref=eps0, stream=stream)
            jumped = float(np.mean([len(r) > 0 for r in p.records()]))
            rows.append({"M": M, "nu": nu.tolist(), "nu_update": nu_upd.tolist(), "final_JT": float(JT[-1]),
                         "jumped_fraction": jumped,
                         "iters_per_s": n_iter * 1000.0 / e0.elapsed_time(e1)})
    logM = np.log(np.array(Ms, dtype=np.float64))
    slopes = [float(np.polyfit(logM, np.log([r["nu"][i] for r in rows]), 1)[0]) for i in range(net.n_ctrl)]
    slopes_upd = [float(np.polyfit(logM, np.log([r["nu_update"][i] for r in rows]), 1)[0])
                  for i in range(net.n_ctrl)]
    big = [i for i, M in enumerate(Ms) if M >= 128]
    slopes_tail = [float(np.polyfit(logM[big], np.log([rows[k]["nu_update"][i] for k in big]), 1)[0])
                   for i in range(net.n_ctrl)]
    line = {"metric": "pulse noise nu_i(M) (Eq. noise) of the accumulated update, fitted exponent of M",
            "value": float(np.mean(slopes_upd)),
            "unit": "exponent b of nu ~ M^b (paper: -1/2)", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic", "dtype": "c64+f64",
            "config": {"workload": f"{wl.name} model, guess amplitude {amp}, {n_iter} iterations, FP32-mixed",
                       "d": wl.d, "nt": wl.nt, "M": Ms},
            "slopes_update": slopes_upd, "slopes_update_M_ge_128": slopes_tail, "slopes_pulse": slopes,
            "runs": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_cross(args, rank, world):
    """Cross-trajectory vs independent-trajectory Krotov on the two-node workload."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    if rank != 0:
        return 0
    from paper_1801_04382_gb300 import Problem, cascaded_chain
    wl = si.CONFIGS["cfg2_d81"]
    n_iter = 20
    net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    eps0 = si.guess_pulses(net.n_ctrl, wl.nt, wl.T, wl.guess_amp)
    S = si.shape_functions(net.n_ctrl, wl.nt, wl.T)
    lam = np.full(net.n_ctrl, wl.lam)
    U = si.uniforms(wl.seed, n_iter + 1, wl.M, wl.draws_per_traj)
    stream = torch.cuda.current_stream()
    out = {}
    for rule in ("independent", "cross"):
        with Problem(net, wl.T, wl.nt, wl.M, eps0, S, lam, U, precision="fp32", stream=stream,
                     update_rule=rule) as p:
            F0 = p.forward(False, stream=stream)
            p.set_profiling(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            JT, _ = p.update(n_iter, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            prof = p.profile()
            out[rule] = {"iters_per_s": n_iter * 1000.0 / e0.elapsed_time(e1), "JT_guess": 1.0 - F0,
                         "JT": [float(x) for x in JT],
                         "kernels": {f"{k}_kernel": {"launches": n, "total_ms": ms, "avg_ms": ms / max(n, 1)}
                                     for k, (ms, n) in prof.items() if n > 0}}
    peaks, _ = measured_peaks()
    fp32_peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    c_ms, c_n = prof["cross"]
    pair_flops = 8.0 * (1 + net.n_ctrl) * wl.M * wl.M * wl.d        # complex MACs of G and A_c per launch
    line = {"metric": "cross-trajectory Krotov (Eq. cross_traj_update) vs independent, iterations/s and J_T",
            "value": out["cross"]["iters_per_s"], "unit": "Krotov iters/s (cross-trajectory update)",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "c64+f64",
            "config": {"workload": f"{wl.name} (d={wl.d}, M={wl.M}, nt={wl.nt}), {n_iter} iterations, FP32-mixed"},
            "independent": out["independent"], "cross": out["cross"],
            "cross_pairs": {"launches": c_n, "avg_ms": c_ms / max(c_n, 1), "flops_per_launch": pair_flops,
                            "tflops": pair_flops / (c_ms / max(c_n, 1) / 1000.0) / 1e12 if c_n else None,
                            "fp32_peak_tflops": fp32_peak}}
    print(json.dumps(line), flush=True)
    return 0


def run_density(args, rank, world):
    """Density-matrix Krotov (Sec. 2.2, Eq. krotovupdate), the convergence reference of the trajectory
    methods, on the two-node chain of the d = 81 workload (T = 50, nt = 1000, seed-free): vec(rho) is
    one state of the four-node Liouville-space network (d^2 = 6561), propagated by the trajectory
    kernels in one CTA per interval.  Iterations/s and the J_T history in FP32-mixed and FP64."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    if rank != 0:
        return 0
    from paper_1801_04382_gb300 import DensityProblem, cascaded_chain
    wl = si.CONFIGS["cfg2_d81"]
    net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    eps0 = si.guess_pulses(net.n_ctrl, wl.nt, wl.T, wl.guess_amp)
    S = si.shape_functions(net.n_ctrl, wl.nt, wl.T)
    lam = np.full(net.n_ctrl, wl.lam)
    stream = torch.cuda.current_stream()
    out = {}
    for prec, n_iter in (("fp32", max(args.steps, 3)), ("fp64", 2)):
        with DensityProblem(net, wl.T, wl.nt, eps0, S, lam, precision=prec, stream=stream) as p:
            F0 = p.forward(False, stream=stream)
            p.update(1, stream=stream)                    # warm-up: captures the iteration graphs
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            JT, _ = p.update(n_iter, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            out[prec] = {"iters_per_s": n_iter * 1000.0 / e0.elapsed_time(e1), "JT_guess": 1.0 - F0,
                         "JT": [float(x) for x in JT], "cheb_terms": p.info.cheb_terms,
                         "liouville_dim": p.info.d}
    line = {"metric": "density-matrix Krotov (Eq. krotovupdate) iterations/s", "value": out["fp32"]["iters_per_s"],
            "unit": "Krotov iters/s (FP32-mixed)", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "dtype": "c64+f64",
            "config": {"workload": f"{wl.name} model as a density matrix (d={wl.d}, Liouville dimension "
                                   f"{wl.d ** 2}, nt={wl.nt}, T={wl.T})"},
            "fp32": out["fp32"], "fp64": out["fp64"],
            "fp32_over_fp64": out["fp32"]["iters_per_s"] / out["fp64"]["iters_per_s"]}
    print(json.dumps(line), flush=True)
    return 0


def oracle_threads() -> int:
    """Threads the oracle's linear algebra runs on: the BLAS pools' sizes where threadpoolctl can
    read them, else the thread-count setting made before numpy loaded."""
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)


def oracle_small_configs():
    """The FP64 oracle, as it stands, on the two smallest workloads at full size (one thread, see
    the top of this file): one Krotov iteration (guess sweep, backward sweep, updating sweep) each,
    as iterations/s and traj.steps/s."""
    from oracle import mcwf
    from oracle import model as om
    out = {}
    cores = oracle_threads()
    for name in ("cfg1_d36", "cfg2_d81"):
        wl = si.CONFIGS[name]
        m = om.build_model(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
        eps = si.guess_pulses(wl.n_nodes, wl.nt, wl.T, wl.guess_amp)
        S = si.shape_functions(wl.n_nodes, wl.nt, wl.T)
        lam = np.full(wl.n_nodes, wl.lam)
        U = si.uniforms(wl.seed, 2, wl.M, wl.draws_per_traj)
        t0 = time.perf_counter()
        mcwf.optimize(m, eps, wl.T, U, S, lam, 1, psi0=m.psi0)
        el = time.perf_counter() - t0
        # the iteration proper is two of the three sweeps timed
        out[name] = {"krotov_iters_per_s": 1.0 / (el * 2.0 / 3.0), "traj_steps_per_s": 3 * wl.M * wl.nt / el,
                     "seconds": el, "cores": cores,
                     "sample": f"full size: d={wl.d}, M={wl.M}, nt={wl.nt}, guess + backward + updating sweep"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl = workload(0)
    steps = []
    base = None
    for _ in range(args.warmup):
        cpu_baseline(wl, budget_s=4.0)
    for _ in range(args.steps):
        base = cpu_baseline(wl, budget_s=8.0)
        steps.append(base["value"])
    value = statistics.median(steps)
    ms = 1000.0 / value
    line = {"metric": METRIC, "value": value, "unit": "Krotov iters/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "d": wl.d, "M": wl.M, "nt": wl.nt},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "Krotov iters/s", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": "Krotov iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world):
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1801_04382_gb300 import Problem, cascaded_chain

    # replicas (default): every rank optimises its own problem (own seed); --shard: the ranks split one
    # problem's trajectories and exchange the update's tile partials over NCCL once per interval
    wl = workload(0 if args.shard else rank, args.precision)
    net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
    n_passes = 2 + args.warmup + args.steps
    eps0 = si.guess_pulses(net.n_ctrl, wl.nt, wl.T, wl.guess_amp)
    S = si.shape_functions(net.n_ctrl, wl.nt, wl.T)
    lam = np.full(net.n_ctrl, wl.lam)
    U = si.uniforms(wl.seed, n_passes, wl.M, wl.draws_per_traj)
    stream = torch.cuda.current_stream()
    shard_kw, M_rank = {}, wl.M
    if args.shard:
        from paper_1801_04382_gb300 import nccl_unique_id, shard_ranges
        from paper_1801_04382_gb300.problem import nccl_library_path
        off, M_rank = shard_ranges(wl.M, world, 1)[rank]
        U = np.ascontiguousarray(U[:, off:off + M_rank])
        shard_kw = dict(traj_offset=off, M_total=wl.M, tile_traj=1)
    # co-state storage from the free device memory (every co-state when they fit)
    prob = Problem(net, wl.T, wl.nt, M_rank, eps0, S, lam, U, precision=wl.precision,
                   ckpt_interval=args.ckpt, stream=stream, **shard_kw)
    if args.shard:
        lib = nccl_library_path()
        uid = [nccl_unique_id(lib) if rank == 0 else None]
        if dist:
            dist.broadcast_object_list(uid, src=0)
        prob.shard_nccl(uid[0], rank, world, lib)
    info = prob.info
    prob.forward(False, stream=stream)                  # guess sweep (pass 0)
    for _ in range(args.warmup):
        prob.update(1, stream=stream)                   # also captures the two iteration graphs

    # ---------------- timed region: K Krotov iterations through the product path (one CUDA graph
    # launch per iteration), inputs resident in HBM
    clk_path = os.path.join(tempfile.gettempdir(), f"kt_clocks_{os.getpid()}.csv")
    proc, fh = clocks_start(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    JT, _ = prob.update(args.steps, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    clocks = clocks_stop(proc, fh, clk_path, local)
    ms_total = reduce_max(ms_total, dist, "cuda")
    ms_step = ms_total / args.steps
    iters_per_s = (1 if args.shard else world) * 1000.0 / ms_step
    traj_steps_per_s = iters_per_s * 2 * wl.M * wl.nt

    # ---------------- per-kernel split: one more iteration launched kernel by kernel, CUDA events on
    # the launching stream around every launch
    prob.set_profiling(True)
    prob.update(1, stream=stream)
    torch.cuda.synchronize()
    prof = prob.profile()
    prob.set_profiling(False)
    prof_ms_iter = sum(ms for ms, _ in prof.values())

    # ---------------- end to end through the public API, host buffers each step
    e2e_steps = max(1, min(args.steps, 3))
    pin = torch.empty((1, M_rank, wl.draws_per_traj), dtype=torch.float64, pin_memory=True)
    host_U = si.uniforms(wl.seed + 7, e2e_steps, M_rank, wl.draws_per_traj)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s_ in range(e2e_steps):
        pin.numpy()[0] = host_U[s_]
        prob.set_uniforms(pin.numpy(), stream=stream)   # H2D: this step's random numbers
        JT_e2e, _ = prob.update(1, stream=stream)        # D2H: J_T (tau_k of all trajectories)
        eps_host = prob.pulses()                         # D2H: the updated pulse
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / e2e_steps
    e2e_ms = reduce_max(e2e_ms, dist, "cuda")
    h2d = M_rank * wl.draws_per_traj * 8
    d2h = (wl.M if args.shard else M_rank) * 16 + net.n_ctrl * wl.nt * 8

    # ---------------- roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    fam = max(prof, key=lambda k: prof[k][0])
    f_ms, f_n = prof[fam]
    avg_s = f_ms / max(f_n, 1) / 1000.0
    nnz = avg_row_nonzeros(net)
    K = info.cheb_terms
    ri = info.threads > 0 and wl.n_cav == 2      # cavity network with real / imaginary coupling classes
    exec_per_elem_term = executed_flops_per_elem_term(nnz, ri)
    survey_per_elem_term = 8.0 * nnz + 12.0      # every coupling counted as a complex multiply-add
    flops_per_launch = exec_per_elem_term * K * wl.d * M_rank
    clk_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = fp32_peak_tflops(clk_max)
    achieved = flops_per_launch / avg_s / 1e12
    s_bytes = 8 if wl.precision == "fp32" else 16
    bytes_per_iter = 5.0 * s_bytes * wl.d * wl.M * wl.nt
    hbm_achieved = bytes_per_iter * (iters_per_s / world) / 1e9
    kernel_bytes = (3 if fam == "fwd" else 2) * s_bytes * wl.d * M_rank
    roof = {"bound": "alu", "kernel": f"{fam}_kernel", "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak,
            "traffic": NCU_TRAFFIC_PER_LAUNCH.get(fam) if wl.precision == "fp32" else None,
            "avg_launch_ms": avg_s * 1e3, "launches": f_n,
            "flops_per_launch": flops_per_launch, "flops_per_elem_term": exec_per_elem_term,
            "flops_per_elem_term_complex_count": survey_per_elem_term,
            "tflops_complex_count": survey_per_elem_term * K * wl.d * M_rank / avg_s / 1e12,
            "algorithmic_bytes_per_launch": kernel_bytes,
            "hbm_gbs_of_kernel": kernel_bytes / avg_s / 1e9,
            "peak_source": f"FP32 FFMA: {sm_count()} SMs x {FP32_LANES} lanes x 2 x {clk_max:.0f} MHz"}
    line = {
        "metric": METRIC, "value": iters_per_s, "unit": "Krotov iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak",
        "vs_baseline": None, "dtype": "c64+f64" if wl.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "d": wl.d, "M": wl.M, "nt": wl.nt, "dt": wl.dt,
                   "precision": "FP32-mixed" if wl.precision == "fp32" else "FP64",
                   "costate_storage": ("every co-state kept" if info.ckpt_interval == 0 else
                                       f"t_0..t_{info.ckpt_kept_prefix} kept, then every {info.ckpt_interval}"),
                   "costate_slots": info.costate_slots, "cheb_terms": K, "tile_traj": info.tile_traj,
                   "threads": info.threads, "l2": "inputs larger than L2 (co-states "
                   f"{info.device_bytes / 1e9:.1f} GB per GPU)",
                   "parallelism": f"trajectory-sharded{world}" if args.shard else f"replicas{world}",
                   "timed_path": "krotov_update: one CUDA graph launch per iteration"},
        "traj_steps_per_s": traj_steps_per_s,
        "hbm_roofline": {"achieved_gbs": hbm_achieved, "peak_gbs": peaks["hbm_gbs"],
                         "frac": hbm_achieved / peaks["hbm_gbs"], "peak_source": peak_src,
                         "bytes_per_iter": bytes_per_iter},
        "final_JT": float(JT[-1]) if JT is not None else None,
        "roofline": roof,
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": "Krotov iters/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "kernels_one_profiled_iteration": {f"{k}_kernel": {"launches": n, "total_ms": ms, "avg_ms": ms / max(n, 1)}
                                           for k, (ms, n) in prof.items() if n > 0},
        "profiled_iteration_ms": prof_ms_iter,
        "gpu_launches": int((prof["fwd"][1] + prof["bwd"][1] + prof["finish"][1] + 4) * args.steps),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_precision_comparison:
        line["fp32_vs_fp64"] = precision_comparison(stream)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
        line["oracle_full_small_configs"] = oracle_small_configs()
    prob.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """Small case of the interval kernels for ncu captures that must stay small.  --profile-d 6561
    (default): the four-node chain, dt = 0.01, M trajectories (--profile-M, default 1024 = the
    benchmark's launch size), 12 intervals.  --profile-d 81: the two-node d = 81 workload (128
    trajectories, nt = 1000, dt = 0.05, FP32-mixed), whose sweeps run as one launch each.  Guess
    sweep, backward sweep, updating forward sweep, with the library's per-launch event timing printed
    at the end.  A few GB on the device at most."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (GB300); the CUDA path has no CPU fallback")
    from paper_1801_04382_gb300 import Problem, cascaded_chain
    if args.profile_d == 81:
        wl = si.CONFIGS["cfg2_d81"]
        nt, T, M = wl.nt, wl.T, wl.M
        net = cascaded_chain(wl.n_nodes, wl.n_cav, wl.delta, wl.g, wl.kappa)
        eps0 = si.guess_pulses(net.n_ctrl, nt, T, wl.guess_amp)
        S = si.shape_functions(net.n_ctrl, nt, T)
        lam = np.full(net.n_ctrl, wl.lam)
        U = si.uniforms(wl.seed, 4, M, wl.draws_per_traj)
    else:
        nt, T, M = 12, 0.12, args.profile_M
        net = cascaded_chain(4, 2)
        eps0 = si.guess_pulses(4, nt, T, 1.0)
        S = si.shape_functions(4, nt, T)
        lam = np.full(4, 10.0)
        U = si.uniforms(4, 4, M, 25)
    with Problem(net, T, nt, M, eps0, S, lam, U, precision=args.precision) as p:
        info = p.info
        print(f"d={info.d} tile_traj={info.tile_traj} threads={info.threads} cheb_terms={info.cheb_terms} "
              f"tiles={info.n_tiles} whole_sweep={info.whole_sweep}")
        p.forward(False)
        p.set_profiling(True)
        p.backward()
        p.forward(True)
        prof = p.profile()
        for k, (ms, n) in prof.items():
            print(f"{k}_kernel: {n} launches, {ms:.3f} ms, {ms / max(n, 1):.4f} ms/launch")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-comparison", action="store_true")
    ap.add_argument("--workload", choices=["cfg5", "mix64", "grad729", "noise", "cross", "profile", "density"],
                    default="cfg5")
    ap.add_argument("--ckpt", type=int, default=-1,
                    help="co-state storage of the cfg5 problem: -1 automatic from free memory (default), "
                         "0 all, K > 0 every K-th")
    ap.add_argument("--profile-M", type=int, default=1024)
    ap.add_argument("--profile-d", type=int, choices=[6561, 81], default=6561)
    ap.add_argument("--shard", action="store_true",
                    help="split one problem's trajectories over the ranks (NCCL exchange of the update's "
                         "partials every interval; strong scaling) instead of one problem per rank")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "mix64":
        return run_mix(args, rank, world)
    if args.workload == "grad729":
        return run_grad(args, rank, world)
    if args.workload == "noise":
        return run_noise(args, rank, world)
    if args.workload == "cross":
        return run_cross(args, rank, world)
    if args.workload == "profile":
        return run_profile(args)
    if args.workload == "density":
        return run_density(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
