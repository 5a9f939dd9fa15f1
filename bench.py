#!/usr/bin/env python
"""Benchmark: Parareal solves/s at 1e-6 relative error against the serial fine
solution, on one B300 (or N independent replicas).

Workload (the PINN-coarse Parareal configuration): European call, K=1,
sigma=0.2, r=0.05, T=1, S in [0, 4] on Nx=1024 points, P=32 slices,
Crank-Nicolson 1024 steps per slice (FP64); coarse propagator = tanh MLP
2->4x64->1 in (S, tau), Xavier init from seed 0, trained 5000 full-batch Adam
steps (lr 1e-3, FP32) on 16384 uniform interior + 1024 boundary/expiry points.

A timed step is one complete Parareal solve through the C ABI: network table
on the grid (one pinn_eval), initial iterate, then fine propagation + fused
correction + increment norm per iteration until the stop rule.  The stop
tolerance is the largest of 1e-6, 3e-7, 1e-7, ... whose result is within 1e-6
of serial fine (checked before timing and after).  Inputs are resident in HBM;
L2 (126 MB) is flushed with a 256 MB write between timed steps, outside the
events.  Also reported: implicit-Euler-coarse Parareal and serial fine on the
same grid, a training step, the fine kernel's roofline, the end-to-end rate
with host buffers, and the oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=1024, P=32, fine_steps=1024, coarse_steps=1)
WIDTHS = [2, 64, 64, 64, 64, 1]
N_INTERIOR, N_BOUNDARY, N_EXPIRY = 16384, 512, 512
TARGET = 1e-6
METRIC = "Parareal solves/s at 1e-6 vs serial fine"
WORKLOAD = ("PINN-coarse Parareal, BS call K=1 sigma=0.2 r=0.05 T=1, Nx=1024 S in [0,4], P=32, "
            "CN 1024 steps/slice FP64, MLP 2->4x64 tanh trained 5k Adam steps on 16384+1024 points")
FLOPS_PER_PT_STEP = 11.0  # CN right-hand side 5 + factored solve 6 (algorithmic, per interior point-step)
# DRAM bytes (read + write) of one fine_propagate launch over the 32 slices of the
# benchmark workload, from one ncu capture per partition (profiles/); a partition
# without a capture of its current code reports null
FINE_TRAFFIC_BYTES = {(2, 4, 4): 425216}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    """One process per GPU (torchrun environment): NCCL on GPUs, gloo on a host
    without them (the CPU tests of this host logic)."""
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(ws, v: float) -> float:
    """The largest of the ranks' values (step time: the job is as slow as its slowest rank)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, ms_per_step: float) -> float:
    """Whole-job solves/s: every rank runs one solve per step (replicas), timed by the slowest."""
    return ws * 1e3 / ms_per_step


def rel_error(U, Uref, P, Nx):
    """max over slices n = 1..P of ||U_n - Uref_n||_2 / ||Uref_n||_2 (harness measurement)."""
    a = U.view(P + 1, Nx)[1:]
    b = Uref.view(P + 1, Nx)[1:]
    return float(((a - b).norm(dim=1) / b.norm(dim=1)).max().item())


def train_network(B, torch, steps, seed=0, prec=None, params=None):
    """The benchmark network: full-batch Adam on the collocation set, BF16 operands on
    the tensor cores (FP32 accumulation, FP64 master weights) unless prec says otherwise;
    params: the problem whose PDE the loss takes (default: the benchmark's)."""
    from paper_2303_03848_b300 import synth

    prec = B.BF16 if prec is None else prec
    cfg = CFG if params is None else params
    X, kind = synth.collocation(seed, N_INTERIOR, N_BOUNDARY, N_EXPIRY, CFG["Smax"], CFG["T"])
    Xd = torch.tensor(X, device="cuda")
    kd = torch.tensor(kind, device="cuda")
    m = B.PinnModel(WIDTHS, [0.0, 0.0], [CFG["Smax"], CFG["T"]], seed=seed)
    loss0 = m.train_step(Xd, kd, cfg, lr=1e-3, prec=prec, want_loss=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timed = min(200, max(steps - 1, 1))
    for i in range(1, steps):
        if i == steps - timed:
            e0.record()
        m.train_step(Xd, kd, cfg, lr=1e-3, prec=prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / timed if steps > 1 else float("nan")
    loss1 = m.train_step(Xd, kd, cfg, lr=1e-3, prec=prec, want_loss=True)
    name = {B.FP64: "fp64", B.FP32: "fp32", B.BF16: "bf16 (tcgen05)"}[prec]
    return m, dict(steps=steps, precision=name, ms_per_step=ms, points=len(kind), loss_first=loss0,
                   loss_last=loss1, points_per_s=len(kind) / (ms * 1e-3) if ms == ms else None)


def choose_tol(prob, kind, model, prec, Uf, B):
    for tol in (1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 1e-10, 1e-11, 0.0):
        U, norms, stats, rc = prob.parareal_solve(kind, model=model, prec=prec, tol=tol)
        err = rel_error(U, Uf, CFG["P"], CFG["Nx"])
        if err <= TARGET:
            return tol, stats[0]["iterations"], err
    return 0.0, CFG["P"], err


def time_solves(prob, kind, model, prec, tol, steps, warmup, torch, flush, graph=True):
    """Device time per solve (CUDA events), L2 flushed between solves.  graph: the
    solve is captured once in a CUDA graph and replayed (one launch per solve);
    otherwise each solve is enqueued by the host loop of parareal_solve."""
    from paper_2303_03848_b300 import binding as B

    g = B.SolveGraph(prob, kind, model=model, prec=prec, tol=tol) if graph else None

    def once():
        if g is not None:
            return g.replay()
        return prob.parareal_solve(kind, model=model, prec=prec, tol=tol, want_stats=False)[0]

    for _ in range(warmup):
        once()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    U = None
    for i in range(steps):
        flush.add_(1.0)  # 256 MB write: evicts L2 between timed steps
        evs[i][0].record()
        U = once()
        evs[i][1].record()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    return ms, U.clone()


def run_ours(args):
    import numpy as np
    import torch

    from paper_2303_03848_b300 import binding as B
    from paper_2303_03848_b300 import build as BUILD

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    BUILD.build()
    prec = B.PREC[args.prec]
    peaks = _peaks()

    t0 = time.perf_counter()
    # the built-in partition rule: deterministic (a tuned choice timed under a
    # profiler could differ), and the autotuner's own pick for this workload
    prob = B.Problem(CFG)
    setup_ms = (time.perf_counter() - t0) * 1e3
    part = prob.partition(0)
    fine_kernel_name = "prop_kernel<M={M},NW={NW},C={C},CN> ({C} CTA cluster per slice)".format(**part)
    fine_traffic = FINE_TRAFFIC_BYTES.get((part["M"], part["NW"], part["C"]))
    model, train = train_network(B, torch, args.train_steps)
    Uf = prob.serial_fine()
    torch.cuda.synchronize()

    tol, iters, err = choose_tol(prob, B.COARSE_PINN, model, prec, Uf, B)
    flush = torch.zeros(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        w0 = time.perf_counter()
        ms, U = time_solves(prob, B.COARSE_PINN, model, prec, tol, args.steps, args.warmup, torch, flush)
        wall = time.perf_counter() - w0
    barrier(ws)
    err_after = rel_error(U, Uf, CFG["P"], CFG["Nx"])
    ms_step = allreduce_max(ws, sum(ms) / len(ms))
    value = job_rate(ws, ms_step)
    ms_direct, _ = time_solves(prob, B.COARSE_PINN, model, prec, tol, 2, 1, torch, flush, graph=False)

    # fine kernel alone: iteration-0 launch shape (all P slices), CUDA events on the current stream
    U0 = Uf.view(CFG["P"] + 1, CFG["Nx"])[:-1].contiguous().view(-1)
    Fo = torch.empty_like(U0)
    for _ in range(2):
        prob.fine_propagate(U0, Fo)
    torch.cuda.synchronize()
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    for a, b in fe:
        a.record()
        prob.fine_propagate(U0, Fo)
        b.record()
    torch.cuda.synchronize()
    fine_ms = statistics.mean(a.elapsed_time(b) for a, b in fe)
    pt_steps = (CFG["Nx"] - 2) * CFG["fine_steps"] * CFG["P"]
    fine_tflops = FLOPS_PER_PT_STEP * pt_steps / (fine_ms * 1e-3) / 1e12
    fp64_peak = 148 * 2 * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12

    # implicit Euler coarse and serial fine on the same grid
    tol_ie, it_ie, err_ie = choose_tol(prob, B.COARSE_IE, None, prec, Uf, B)
    ms_ie, _ = time_solves(prob, B.COARSE_IE, None, prec, tol_ie, max(2, args.steps // 2), 1, torch, flush)
    sf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
    for a, b in sf:
        a.record()
        prob.serial_fine(Uf)
        b.record()
    torch.cuda.synchronize()
    serial_ms = statistics.mean(a.elapsed_time(b) for a, b in sf)

    # per-precision network tables at the same accuracy target; the coarse output's
    # error against FP64 is the table u_theta(S_j, tau_n) on the solve's grid
    S = torch.linspace(0.0, CFG["Smax"], CFG["Nx"], dtype=torch.float64, device="cuda")
    tau = torch.linspace(0.0, CFG["T"], CFG["P"] + 1, dtype=torch.float64, device="cuda")
    Xg = torch.stack(torch.meshgrid(S, tau, indexing="xy"), dim=-1).reshape(-1, 2).contiguous()
    u64 = model.eval(Xg, prec=B.FP64)
    per_prec = {}
    for name, p in B.PREC.items():
        tl, itp, ep = choose_tol(prob, B.COARSE_PINN, model, p, Uf, B)
        msp, _ = time_solves(prob, B.COARSE_PINN, model, p, tl, 2, 1, torch, flush)
        up = model.eval(Xg, prec=p)
        cerr = ((up - u64).abs().max() / u64.abs().max()).item()
        per_prec[name] = dict(tol=tl, iterations=itp, err_vs_serial_fine=ep, ms_per_solve=statistics.mean(msp),
                              coarse_err_vs_fp64=cerr)

    # one solve by phase (CUDA events on graph-replayed solves): solves stopped after
    # one and after two iterations give the cost of an iteration (fine propagation,
    # fused correction and stop test) and the fixed part (network table, initial
    # iterate, result copy); the table alone is timed as one evaluation on the grid
    def replay_ms(graph, reps=3):
        graph.replay()
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            graph.replay()
            b.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return min(out)

    g1 = B.SolveGraph(prob, B.COARSE_PINN, model=model, prec=prec, tol=0.0, max_iter=1)
    g2 = B.SolveGraph(prob, B.COARSE_PINN, model=model, prec=prec, tol=0.0, max_iter=2)
    t1, t2 = replay_ms(g1), replay_ms(g2)
    del g1, g2
    model.eval(Xg, prec=prec)
    tab = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        model.eval(Xg, prec=prec)
        b.record()
        torch.cuda.synchronize()
        tab.append(a.elapsed_time(b))
    phases = {"per_iteration_ms": t2 - t1, "fixed_ms": 2 * t1 - t2, "network_table_ms": min(tab),
              "iterations": iters, "solve_ms": ms_step,
              "note": "solve = fixed + iterations x per_iteration; the fixed part holds the table"}

    # end to end through the C ABI with host buffers
    w_host = torch.tensor(model.get_weights()).pin_memory()
    U_host = torch.empty(prob.total_state, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        model.set_weights(w_host.numpy())
        Ud, *_ = prob.parareal_solve(B.COARSE_PINN, model=model, prec=prec, tol=tol, want_stats=False)
        U_host.copy_(Ud, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - s0) * 1e3)
    e2e_step = allreduce_max(ws, statistics.mean(e2e_ms))

    # the single-GPU context legs and the CPU baseline run at N = 1 only (at N > 1
    # every rank would hold its GPU meanwhile, and the baseline belongs to rank 0 at N = 1)
    batched = pinn = train3 = cpu = None
    if ws == 1:
        batched = batched_leg(B, torch) if args.batched else None
        pinn = pinn_leg(B, torch)
        train3 = train_leg(B, torch)
        cpu = cpu_baseline(model.get_weights(), iters, budget_s=args.cpu_seconds)

    if rank != 0:
        return
    kmax = CFG["P"]
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "coarse": "pinn", "pinn_precision": args.prec, "tol": tol,
                   "iterations": iters, "err_vs_serial_fine": err_after, "l2_flush": "256 MB write between steps",
                   "launch": "whole solve captured in one CUDA graph, replayed per step",
                   "ms_per_solve_host_loop": statistics.mean(ms_direct),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "e2e": {"value": job_rate(ws, e2e_step), "unit": "solves/s", "h2d_bytes_per_step": 8 * model.n_params,
                "d2h_bytes_per_step": 8 * prob.total_state},
        # network table (grid points, weight pack for the tensor-core path, evaluation, Dirichlet fix),
        # initial iterate, per iteration fine propagation + stop test, result copy
        "gpu_launches": (4 if prec == B.BF16 else 3) + 1 + 2 * kmax + 1,
        "roofline": {"bound": "alu", "achieved": fine_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": fine_tflops / fp64_peak, "traffic": fine_traffic, "kernel": fine_kernel_name,
                     "peak_note": "FP64: 148 SM x 2 DFMA lanes/clk (measured) x 2 flop x max SM clock"},
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "fine_kernel": {"ms": fine_ms, "grid_pt_steps_per_s": pt_steps / (fine_ms * 1e-3)},
        # iteration k (0-based) propagates slices k..P-1: executed = (Nx-2) M_f sum_k (P-k),
        # useful = (Nx-2) M_f P (what serial fine does once)
        "grid_pt_steps": grid_pt_steps(iters, value),
        "ie_coarse": {"tol": tol_ie, "iterations": it_ie, "err_vs_serial_fine": err_ie,
                      "solves_per_s": 1e3 / statistics.mean(ms_ie)},
        "serial_fine_ms": serial_ms,
        "speedup_vs_serial_fine": {"pinn": serial_ms / ms_step, "ie": serial_ms / statistics.mean(ms_ie)},
        "phases": phases,
        "per_precision": per_prec,
        "train_step": train,
        "batched": batched,
        "pinn_eval": pinn,
        "train_2x6x128": train3,
        "setup_ms": setup_ms,
        "partition": dict(part, chosen_by="built-in rule (the autotuner picks the same on this workload)"),
        "wall_s_timed": wall,
    }
    print(json.dumps(out), flush=True)


def run_fine_only(args):
    """The fine kernel alone: fine_propagate over all P slices of the workload (no training, no solve)."""
    import torch

    from paper_2303_03848_b300 import binding as B
    from paper_2303_03848_b300 import build as BUILD

    BUILD.build()
    prob = B.Problem(CFG)
    Uf = prob.serial_fine()
    U0 = Uf.view(CFG["P"] + 1, CFG["Nx"])[:-1].contiguous().view(-1)
    Fo = torch.empty_like(U0)
    for _ in range(args.warmup):
        prob.fine_propagate(U0, Fo)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        a.record()
        prob.fine_propagate(U0, Fo)
        b.record()
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    pt = (CFG["Nx"] - 2) * CFG["fine_steps"] * CFG["P"]
    print(json.dumps({"mode": "fine", "ms": ms, "grid_pt_steps_per_s": pt / (ms * 1e-3),
                      "tflops_algorithmic": FLOPS_PER_PT_STEP * pt / (ms * 1e-3) / 1e12}), flush=True)


def batched_leg(B, torch, n_inst=4096, solve=True, rule_too=False, pinn_solve=False, cpu_seconds=10.0):
    """Batched workload: n_inst instances (K, sigma, r, T, Nx seeded), P=64, CN 256 steps/slice.

    The partition of every grid size is picked by the autotuner
    (bs_problem_init_tuned).  Times fine_propagate over every slice of every
    instance (one launch per partition class) and, optionally, one
    implicit-Euler-coarse Parareal solve of the whole batch at tol 1e-6.
    rule_too: also time the built-in partition rule for comparison.
    cpu_seconds: budget of the oracle's all-core sample of the IE solve (0: none).
    pinn_solve: also one Parareal solve of the batch with the parametric network
    5->6x128 (BF16 table) as coarse propagator, and both solves' error against
    the batch's serial fine solution.
    """
    from paper_2303_03848_b300 import synth

    insts = synth.batched_instances(0, n_inst, P=64, fine_steps=256, coarse_steps=1)
    pt = sum((p["Nx"] - 2) * p["fine_steps"] * p["P"] for p in insts)
    peak = 148 * 2 * 2 * float(_peaks().get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)

    def time_fine(prob):
        Uin = torch.rand(prob.total_slice, dtype=torch.float64, device="cuda", generator=gen)
        Fo = torch.empty_like(Uin)
        prob.fine_propagate(Uin, Fo)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        for a, b in ev:
            a.record()
            prob.fine_propagate(Uin, Fo)
            b.record()
        torch.cuda.synchronize()
        assert prob.device_status() == B.BS_OK
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    out = {"instances": n_inst, "P": 64, "fine_steps": 256, "Nx": "uniform over 256..4096"}
    if rule_too:
        rule = B.Problem(insts)
        ms = time_fine(rule)
        out["rule_partition"] = {"fine_ms": ms, "fine_frac_of_fp64_peak": FLOPS_PER_PT_STEP * pt / (ms * 1e-3) / 1e12 / peak,
                                 "partitions": sorted({(p["Nx"], tuple(rule.partition(i).values()))
                                                       for i, p in enumerate(insts)})}
        rule.close()
        torch.cuda.empty_cache()
    t0 = time.perf_counter()
    prob = B.Problem(insts, tuned=True)
    setup_s = time.perf_counter() - t0
    ms = time_fine(prob)
    tf = FLOPS_PER_PT_STEP * pt / (ms * 1e-3) / 1e12
    chosen = {r["Nx"]: "M=%d NW=%d C=%d S2=%d" % (r["M"], r["NW"], r["C"], r["S2"]) for r in prob.tuning if r["chosen"]}
    out.update({"setup_s_with_tuning": setup_s, "tuned_partitions": {str(k): v for k, v in sorted(chosen.items())},
                "candidates_timed": len(prob.tuning),
                "fine_ms": ms, "grid_pt_steps_per_s": pt / (ms * 1e-3),
                "fine_tflops_algorithmic": tf, "fine_frac_of_fp64_peak": tf / peak})
    torch.cuda.empty_cache()
    if solve:
        # statistics from one direct call, time from replays of the whole batched
        # solve captured as one CUDA graph (persistent propagation launches inside)
        U, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=1e-6, max_iter=64)
        its = [st["iterations"] for st in stats]
        del U
        g = B.SolveGraph(prob, B.COARSE_IE, tol=1e-6, max_iter=64)
        reps = []
        for _ in range(2):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            g.replay()
            s1.record()
            torch.cuda.synchronize()
            reps.append(s0.elapsed_time(s1))
        ms_solve = min(reps)
        out.update({"ie_solve_ms": ms_solve, "ie_solves_per_s": n_inst / (ms_solve * 1e-3),
                    "ie_launch": "whole batched solve in one CUDA graph",
                    "ie_iterations_mean": float(sum(its)) / len(its), "ie_iterations_max": max(its),
                    "ie_status": rc})
        if cpu_seconds > 0:
            out["ie_cpu_baseline"] = batched_cpu_baseline(insts, budget_s=cpu_seconds)
        del g
        if pinn_solve:
            Uf = prob.serial_fine()

            def batch_error(U):
                worst = 0.0
                for i, p in enumerate(insts):
                    o, P, Nx = prob.state_off[i], p["P"], p["Nx"]
                    a = U[o + Nx:o + (P + 1) * Nx].view(P, Nx)
                    b = Uf[o + Nx:o + (P + 1) * Nx].view(P, Nx)
                    worst = max(worst, float(((a - b).norm(dim=1) / b.norm(dim=1)).max()))
                return worst

            U, _, _, _ = prob.parareal_solve(B.COARSE_IE, tol=1e-6, max_iter=64, want_stats=False)
            out["ie_err_vs_serial_fine"] = batch_error(U)
            del U
            net, tr = train_parametric(B, torch)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            U, norms, stats, rc = prob.parareal_solve(B.COARSE_PINN, model=net, prec=B.BF16, tol=1e-6, max_iter=64)
            s1.record()
            torch.cuda.synchronize()
            pits = [st["iterations"] for st in stats]
            pms = s0.elapsed_time(s1)
            out["pinn_coarse"] = {"network": "5->6x128 tanh->1, BF16 table on the tensor cores", "training": tr,
                                  "solve_ms": pms, "solves_per_s": n_inst / (pms * 1e-3), "tol": 1e-6,
                                  "iterations_mean": float(sum(pits)) / len(pits), "iterations_max": max(pits),
                                  "err_vs_serial_fine": batch_error(U), "status": rc,
                                  "launch": "direct call (host loop over iterations)"}
            del U, Uf
    prob.close()
    torch.cuda.empty_cache()
    return out


def train_parametric(B, torch, steps=300, n_points=65536):
    """The batched workload's coarse network 5->6x128 tanh on (S, tau, sigma, r, K):
    BF16 full-batch Adam on seeded collocation points over the batch's parameter box."""
    from paper_2303_03848_b300 import synth

    widths = [5] + [128] * 6 + [1]
    lo, hi = [0.0, 0.0, 0.1, 0.0, 0.5], [8.0, 2.0, 0.5, 0.08, 2.0]
    nb = n_points // 32
    X, kind = synth.collocation_parametric(1, n_points - 2 * nb, nb, nb, 4.0, 2.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=2.0, Smax=8.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    net = B.PinnModel(widths, lo, hi, seed=0)
    first = net.train_step(Xd, kd, prob, lr=1e-3, smax_over_K=4.0, prec=B.BF16, want_loss=True)
    for _ in range(steps - 2):
        net.train_step(Xd, kd, prob, lr=1e-3, smax_over_K=4.0, prec=B.BF16)
    last = net.train_step(Xd, kd, prob, lr=1e-3, smax_over_K=4.0, prec=B.BF16, want_loss=True)
    return net, {"steps": steps, "points": len(kind), "precision": "bf16 (tcgen05)", "loss_first": first,
                 "loss_last": last}


def pinn_leg(B, torch, n_points=1 << 24):
    """Network evaluation throughput: the batched workload's 5->6x128 network on n_points points."""
    from paper_2303_03848_b300 import synth

    widths = [5] + [128] * 6 + [1]
    lo, hi = [0.0, 0.0, 0.1, 0.0, 0.5], [8.0, 2.0, 0.5, 0.08, 2.0]
    m = B.PinnModel(widths, lo, hi, seed=0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    X = torch.rand(n_points, 5, dtype=torch.float64, device="cuda", generator=gen)
    X = X * (torch.tensor(hi, device="cuda", dtype=torch.float64) - torch.tensor(lo, device="cuda", dtype=torch.float64)) \
        + torch.tensor(lo, device="cuda", dtype=torch.float64)
    flops_pt = 2 * sum(widths[l] * widths[l - 1] for l in range(1, len(widths)))
    tensor_flops_pt = 2 * 5 * 128 * 128
    tanh_pt = 6 * 128
    mhz = float(_peaks().get("sm_max_mhz", 2032.0))
    mufu_peak = 148 * 16 * mhz * 1e6  # tanh.approx.f32: 16 per clock per SM (measured)
    bf16_peak = float(_peaks().get("bf16_tflops", 1754.7))
    out = {"network": "5->6x128 tanh->1", "points": n_points}
    for name, prec in (("fp64", B.FP64), ("fp32", B.FP32), ("bf16", B.BF16)):
        n = n_points if name != "fp64" else n_points // 16
        Xn = X[:n].contiguous()
        m.eval(Xn, prec=prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            m.eval(Xn, prec=prec)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 3
        pps = n / (ms * 1e-3)
        rec = {"ms": ms, "points": n, "points_per_s": pps, "tflops_algorithmic": flops_pt * pps / 1e12}
        if name == "bf16":
            rec.update({"path": "tcgen05 (hidden 128x128 layers), FP32 accumulation in TMEM",
                        "tensor_tflops": tensor_flops_pt * pps / 1e12,
                        "tensor_frac_of_bf16_peak": tensor_flops_pt * pps / 1e12 / bf16_peak,
                        "tanh_per_s": tanh_pt * pps, "tanh_frac_of_mufu_peak": tanh_pt * pps / mufu_peak})
        out[name] = rec
    assert m.device_status() == B.BS_OK
    return out


def train_leg(B, torch, n_points=65536, steps=20):
    """Training throughput: 2->6x128 tanh network, 65536 collocation points (15/16
    interior uniform in [0,4]x[0,1], 1/16 boundary and expiry), one full-batch Adam
    step = forward with the four derivative streams, loss, adjoint, weight gradient."""
    from paper_2303_03848_b300 import synth

    widths = [2] + [128] * 6 + [1]
    n_b = n_points // 32
    X, kind = synth.collocation(0, n_points - 2 * n_b, n_b, n_b, 4.0, 1.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    # algorithmic flops per point: forward 4 streams through every layer GEMM,
    # adjoint 4 streams back, weight gradient 4 streams: 3 x 4 x 2 x sum(w_in w_out)
    gemm = sum(widths[l] * widths[l - 1] for l in range(1, len(widths)))
    flops_pt = 3 * 4 * 2 * gemm
    out = {"network": "2->6x128 tanh->1", "points": len(kind)}
    for name, prec in (("fp32", B.FP32), ("bf16", B.BF16)):
        m = B.PinnModel(widths, [0.0, 0.0], [4.0, 1.0], seed=0)
        first = sum(m.train_step(Xd, kd, prob, lr=1e-3, prec=prec, want_loss=True))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            m.train_step(Xd, kd, prob, lr=1e-3, prec=prec)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        last = sum(m.train_step(Xd, kd, prob, lr=1e-3, prec=prec, want_loss=True))
        pps = len(kind) / (ms * 1e-3)
        out[name] = {"ms_per_step": ms, "points_per_s": pps, "tflops_algorithmic": flops_pt * pps / 1e12,
                     "loss_first": first, "loss_after": last, "steps": steps + 2}
    # the tensor-core step is bound by HBM traffic: per hidden layer the stored
    # (z_0, z_1, z_2, z_3) in FP16 (layer 1: t only, FP32) written by the forward and
    # read by the adjoint, and the BF16 h and dz operand blocks (4 streams) written
    # once and read once by the weight gradient; per point the inputs (read by the
    # forward and by the adjoint's input-layer gradient) and the kinds
    w, nh, n = widths[1], len(widths) - 2, len(kind)
    act = (8 * (nh - 1) + 4) * 2
    blocks = 8 * (nh - 1) * 2 * 2
    per_point = 2 * 16 + 1
    hbm = n * (w * (act + blocks) + per_point)
    peak = _peaks().get("hbm_gbs")
    ach = hbm / (out["bf16"]["ms_per_step"] * 1e-3) / 1e9
    out["bf16"]["roofline"] = {"bound": "hbm", "algorithmic_bytes_per_step": hbm, "achieved": ach, "peak": peak,
                               "unit": "GB/s", "frac": ach / peak if peak else None,
                               "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    return out


def generalize_leg(B, torch, train_steps, sigmas=(0.2, 0.3, 0.4, 0.5), rs=(0.01, 0.03, 0.05),
                   tols=(1e-2, 1e-3, 1e-4, 1e-6)):
    """Parameter generalisation (the analogue of the paper's Fig. 4): the benchmark network
    (2->4x64 on (S, tau)) trained at sigma = 0.4, r = 0.03 is the coarse propagator of
    benchmark-grid instances at other (sigma, r).  Per instance: the network table's own
    error against serial fine, and per tolerance the iterations and error of the
    network-coarse and of the implicit-Euler-coarse solve."""
    trained = dict(CFG, sigma=0.4, r=0.03)
    model, tr = train_network(B, torch, train_steps, params=trained)
    S = torch.linspace(0.0, CFG["Smax"], CFG["Nx"], dtype=torch.float64, device="cuda")
    tau = torch.linspace(0.0, CFG["T"], CFG["P"] + 1, dtype=torch.float64, device="cuda")
    Xg = torch.stack(torch.meshgrid(S, tau, indexing="xy"), dim=-1).reshape(-1, 2).contiguous()
    table = model.eval(Xg, prec=B.BF16)
    rows = []
    for sigma in sigmas:
        for r in rs:
            cfg = dict(CFG, sigma=sigma, r=r)
            prob = B.Problem(cfg)
            Uf = prob.serial_fine()
            row = {"sigma": sigma, "r": r, "table_err_vs_serial_fine": rel_error(table, Uf, CFG["P"], CFG["Nx"])}
            for name, kind, mdl in (("pinn", B.COARSE_PINN, model), ("ie", B.COARSE_IE, None)):
                row[name] = []
                for tol in tols:
                    U, _, stats, rc = prob.parareal_solve(kind, model=mdl, prec=B.BF16, tol=tol, max_iter=CFG["P"])
                    row[name].append({"tol": tol, "iterations": stats[0]["iterations"],
                                      "err_vs_serial_fine": rel_error(U, Uf, CFG["P"], CFG["Nx"]), "status": rc})
            rows.append(row)
            prob.close()
    return {"mode": "generalize", "grid": "Nx=1024, S in [0,4], K=1 T=1, P=32, 1024 CN steps per slice",
            "network": "2->4x64 tanh, BF16 table", "trained_at": {"sigma": 0.4, "r": 0.03}, "training": tr,
            "rows": rows}


def data_coarse_leg(B, torch, train_steps, tols=(1e-2, 1e-3, 1e-4, 1e-6)):
    """Data-only coarse network (Section 4 trains one on fine-propagator output,
    without the PDE terms, next to the PINN): the benchmark network trained on
    the serial fine solution at every grid point of the benchmark workload (kind-4
    data points), against the PINN trained as usual; per coarse propagator the
    table's error against serial fine and, per tolerance, iterations and error."""
    prob = B.Problem(CFG)
    Uf = prob.serial_fine()
    S = torch.linspace(0.0, CFG["Smax"], CFG["Nx"], dtype=torch.float64, device="cuda")
    tau = torch.linspace(0.0, CFG["T"], CFG["P"] + 1, dtype=torch.float64, device="cuda")
    Xg = torch.stack(torch.meshgrid(S, tau, indexing="xy"), dim=-1).reshape(-1, 2).contiguous()
    kd = torch.full((Xg.shape[0],), 4, dtype=torch.int8, device="cuda")
    dnet = B.PinnModel(WIDTHS, [0.0, 0.0], [CFG["Smax"], CFG["T"]], seed=0)
    loss0 = dnet.train_step(Xg, kd, CFG, lr=1e-3, prec=B.BF16, want_loss=True, y=Uf)
    for _ in range(1, train_steps):
        dnet.train_step(Xg, kd, CFG, lr=1e-3, prec=B.BF16, y=Uf)
    loss1 = dnet.train_step(Xg, kd, CFG, lr=1e-3, prec=B.BF16, want_loss=True, y=Uf)
    pinn, tr = train_network(B, torch, train_steps)
    out = {"mode": "datacoarse", "grid": "Nx=1024, S in [0,4], K=1 sigma=0.2 r=0.05 T=1, P=32, 1024 CN steps per slice",
           "network": "2->4x64 tanh, BF16 table",
           "data_training": {"points": int(Xg.shape[0]), "steps": train_steps, "precision": "bf16 (tcgen05)",
                             "data_mse_first": loss0[0], "data_mse_last": loss1[0]},
           "pinn_training": tr, "coarse": {}}
    for name, kind, mdl in (("data-nn", B.COARSE_PINN, dnet), ("pinn", B.COARSE_PINN, pinn), ("ie", B.COARSE_IE, None)):
        row = {}
        if mdl is not None:
            row["table_err_vs_serial_fine"] = rel_error(mdl.eval(Xg, prec=B.BF16), Uf, CFG["P"], CFG["Nx"])
        row["solves"] = []
        for tol in tols:
            U, _, stats, rc = prob.parareal_solve(kind, model=mdl, prec=B.BF16, tol=tol, max_iter=CFG["P"])
            row["solves"].append({"tol": tol, "iterations": stats[0]["iterations"],
                                  "err_vs_serial_fine": rel_error(U, Uf, CFG["P"], CFG["Nx"]), "status": rc})
        out["coarse"][name] = row
    return out


def sweep_leg(B, torch, model, Ps=(4, 8, 16, 32, 64), total_steps=32768):
    """Speedup against P on one GPU next to the bound of Eq. 8 (the paper's Figs. 5-6):
    the benchmark grid with a fixed total of fine steps split over P slices; per P the
    serial fine time, and per coarse propagator the iterations and time to 1e-6 against
    serial fine (graph-replayed solves), the speedup, and the bound
    1 / ((1 + K/P) c_c/c_f + K/P) with c_c, c_f the measured coarse and fine
    propagation times of one slice (all slices side by side)."""
    from paper_2303_03848_b300 import binding as BB

    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            a, b = ev()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return min(out)

    flush = torch.zeros(1, dtype=torch.float64, device="cuda")
    rows = []
    for P in Ps:
        cfg = dict(CFG, P=P, fine_steps=total_steps // P)
        prob = BB.Problem(cfg)
        Uf = prob.serial_fine()
        serial_ms = timed(lambda: prob.serial_fine(Uf))
        U0 = Uf.view(P + 1, cfg["Nx"])[:-1].contiguous().view(-1)
        Fo = torch.empty_like(U0)
        c_f = timed(lambda: prob.fine_propagate(U0, Fo))
        c_c = timed(lambda: prob.coarse_propagate(U0, Fo))
        row = {"P": P, "fine_steps_per_slice": cfg["fine_steps"], "serial_fine_ms": serial_ms, "c_f_ms": c_f,
               "c_c_ms": c_c}
        for name, kind, mdl in (("ie", BB.COARSE_IE, None), ("pinn", BB.COARSE_PINN, model)):
            tol = None
            for cand in (1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 0.0):
                U, norms, stats, rc = prob.parareal_solve(kind, model=mdl, prec=BB.BF16, tol=cand)
                err = rel_error(U, Uf, P, cfg["Nx"])
                if err <= TARGET:
                    tol, K = cand, stats[0]["iterations"]
                    break
            ms, _ = time_solves(prob, kind, mdl, BB.BF16, tol, 3, 2, torch, flush)
            ms = statistics.mean(ms)
            bound = 1.0 / ((1.0 + K / P) * (c_c / c_f) + K / P)
            row[name] = {"tol": tol, "iterations": K, "ms": ms, "speedup": serial_ms / ms, "eq8_bound": bound,
                         "parallel_efficiency": serial_ms / ms / P}
        rows.append(row)
        prob.close()
    return {"grid": "Nx=1024, S in [0,4], K=1 sigma=0.2 r=0.05 T=1", "total_fine_steps": total_steps, "rows": rows}


def run_large(args):
    """Large single instance: Nx=65536, S in [0,8], sigma 0.3, r 0.03, T 2, K 1, P=256, CN 4096 steps/slice."""
    import torch

    from paper_2303_03848_b300 import binding as B
    from paper_2303_03848_b300 import build as BUILD

    BUILD.build()
    cfg = dict(K=1.0, sigma=0.3, r=0.03, T=2.0, Smax=8.0, Nx=65536, P=args.large_p, fine_steps=args.large_steps,
               coarse_steps=1)
    prob = B.Problem(cfg)
    part = dict(prob.partition(0), slices_per_cta=prob.slices_per_cta(0))
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    a, b = ev()
    a.record()
    Uf = prob.serial_fine()
    b.record()
    torch.cuda.synchronize()
    serial_ms = a.elapsed_time(b)
    U0 = Uf.view(cfg["P"] + 1, cfg["Nx"])[:-1].contiguous().view(-1)
    Fo = torch.empty_like(U0)
    prob.fine_propagate(U0, Fo)  # warm-up
    a, b = ev()
    a.record()
    prob.fine_propagate(U0, Fo)
    b.record()
    torch.cuda.synchronize()
    fine_ms = a.elapsed_time(b)
    pt = (cfg["Nx"] - 2) * cfg["fine_steps"] * cfg["P"]
    tf = FLOPS_PER_PT_STEP * pt / (fine_ms * 1e-3) / 1e12
    peak = 148 * 2 * 2 * float(_peaks().get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
    # implicit-Euler coarse Parareal to 1e-8 against serial fine: the loosest
    # device tolerance (increment norm) that reaches it, each candidate solve timed
    target = 1e-8
    for ie_tol in (1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 1e-10, 0.0):
        a, b = ev()
        a.record()
        U, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=ie_tol, max_iter=cfg["P"])
        b.record()
        torch.cuda.synchronize()
        err = rel_error(U, Uf, cfg["P"], cfg["Nx"])
        ie_ms = a.elapsed_time(b)
        if err <= target:
            break
    # the network coarse propagator of this workload: 2->8x256 tanh, BF16 on the
    # tensor cores, evaluated on the (P+1) x Nx grid (the table one solve needs);
    # under a state-independent coarse propagator the solve itself needs k = P
    widths = [2] + [256] * 8 + [1]
    net = B.PinnModel(widths, [0.0, 0.0], [cfg["Smax"], cfg["T"]], seed=0)
    S = torch.linspace(0.0, cfg["Smax"], cfg["Nx"], dtype=torch.float64, device="cuda")
    tau = torch.linspace(0.0, cfg["T"], cfg["P"] + 1, dtype=torch.float64, device="cuda")
    Xg = torch.stack([S.repeat(cfg["P"] + 1), tau.repeat_interleave(cfg["Nx"])], dim=1).contiguous()
    net.eval(Xg, prec=B.BF16)
    a, b = ev()
    a.record()
    net.eval(Xg, prec=B.BF16)
    b.record()
    torch.cuda.synchronize()
    table_ms = a.elapsed_time(b)
    flops_pt = 2 * sum(widths[l] * widths[l - 1] for l in range(1, len(widths)))
    pinn = {"network": "2->8x256 tanh->1", "points": Xg.shape[0], "bf16_table_ms": table_ms,
            "points_per_s": Xg.shape[0] / (table_ms * 1e-3),
            "tensor_tflops": 7 * 2 * 256 * 256 * Xg.shape[0] / (table_ms * 1e-3) / 1e12,
            "tflops_algorithmic": flops_pt * Xg.shape[0] / (table_ms * 1e-3) / 1e12,
            "status": net.device_status()}
    # the oracle on one host core: consecutive slices of serial fine for about
    # cpu_seconds, extrapolated to all P slices
    cpu = None
    if args.cpu_seconds > 0:
        import oracle as orc

        op = orc.params(**cfg)
        V = orc.payoff(op)
        n_done, t0 = 0, time.perf_counter()
        while n_done < cfg["P"] and (n_done == 0 or time.perf_counter() - t0 < args.cpu_seconds):
            V = orc.fine(op, n_done, V)
            n_done += 1
        t_cpu = time.perf_counter() - t0
        rate = (cfg["Nx"] - 2) * cfg["fine_steps"] * n_done / t_cpu
        cpu = {"value": rate, "unit": "grid-pt-steps/s", "cores": 1, "kind": "oracle", **host_cpu(),
               "serial_fine_s_extrapolated": t_cpu * cfg["P"] / n_done,
               "sample": f"the oracle's serial fine, first {n_done} of {cfg['P']} slices ({t_cpu:.1f} s); "
                         f"serial fine time extrapolated by slice count"}
    print(json.dumps({"mode": "large", "config": cfg, "partition": part, "serial_fine_ms": serial_ms,
                      "fine_ms": fine_ms, "grid_pt_steps_per_s": pt / (fine_ms * 1e-3), "fine_tflops_algorithmic": tf,
                      "fine_frac_of_fp64_peak": tf / peak, "ie_target": target, "ie_tol": ie_tol, "ie_solve_ms": ie_ms,
                      "ie_iterations": stats[0]["iterations"], "ie_err_vs_serial_fine": err,
                      "speedup_vs_serial_fine": serial_ms / ie_ms, "status": rc, "pinn_coarse_table": pinn,
                      "cpu_baseline": cpu}),
          flush=True)


def grid_pt_steps(iters, solves_per_s):
    per_slice = (CFG["Nx"] - 2) * CFG["fine_steps"]
    P = CFG["P"]
    executed = per_slice * sum(P - k for k in range(iters))
    useful = per_slice * P
    return {"executed_per_solve": executed, "useful_per_solve": useful,
            "executed_per_s": executed * solves_per_s, "useful_per_s": useful * solves_per_s}


def host_cpu():
    """CPU model and logical core count of the host the baseline runs on."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "host_cores": os.cpu_count()}


def batched_cpu_baseline(insts, budget_s=10.0, tol=1e-6):
    """The oracle on all host cores for the batched implicit-Euler-coarse solve.

    Worker threads (the oracle is C called through ctypes, which releases the
    GIL) take the batch's seeded instances in order and run the oracle's
    Parareal to tol until budget_s has passed; the whole batch's time is
    extrapolated from the instances finished by their share of sum (Nx - 2).
    """
    import threading

    import oracle as orc

    orc.build()
    cores = os.cpu_count() or 1
    lock = threading.Lock()
    state = {"next": 0, "done": [], "iters": []}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                i = state["next"]
                if i >= len(insts) or time.perf_counter() - t0 > budget_s:
                    return
                state["next"] = i + 1
            p = insts[i]
            _, norms, _ = orc.parareal(orc.params(**p), orc.COARSE_IE, tol=tol, max_iter=p["P"])
            with lock:
                state["done"].append(i)
                state["iters"].append(len(norms))

    th = [threading.Thread(target=worker) for _ in range(cores)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    wall = time.perf_counter() - t0
    done = state["done"]
    w_done = sum(insts[i]["Nx"] - 2 for i in done)
    w_all = sum(p["Nx"] - 2 for p in insts)
    t_full = wall * w_all / w_done
    return {"value": len(insts) / t_full, "unit": "solves/s", "cores": cores, "kind": "oracle", **host_cpu(),
            "sample": f"implicit-Euler-coarse Parareal to {tol:g} on the first {len(done)} of the {len(insts)} "
                      f"seeded instances ({wall:.1f} s on {cores} threads); batch time extrapolated by "
                      f"sum (Nx - 2)", "iterations_mean": float(sum(state["iters"])) / len(done)}


def cpu_baseline(weights, iters, budget_s=20.0):
    """The oracle, as it stands, on the host: one Parareal-PINN iteration per sample."""
    import numpy as np

    import oracle as orc

    p = orc.params(**CFG)
    m = orc.MLP(WIDTHS, weights, [0.0, 0.0], [CFG["Smax"], CFG["T"]])
    t0 = time.perf_counter()
    g = orc.pinn_table(p, m)
    t_table = time.perf_counter() - t0
    done = 0
    t1 = time.perf_counter()
    while True:
        done += 1
        orc.parareal(p, orc.COARSE_PINN, g=g, tol=0.0, max_iter=done)
        if time.perf_counter() - t1 > budget_s or done >= iters:
            break
    # parareal(max_iter=k) reruns iterations 0..k-1; total work sum_{k<=done} k iterations
    t_all = time.perf_counter() - t1
    work = done * (done + 1) / 2
    t_iter = t_all / work
    t_solve = t_table + iters * t_iter
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle", **host_cpu(),
            "sample": f"network table + Parareal iterations 1..{done} of the same workload, "
                      f"per-iteration time extrapolated to the {iters} iterations the solve needs"}


def run_reference(args):
    import numpy as np

    import oracle as orc
    from paper_2303_03848_b300 import synth

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    orc.build()
    p = orc.params(**CFG)
    m = orc.MLP(WIDTHS, synth.xavier_params(WIDTHS, 0), [0.0, 0.0], [CFG["Smax"], CFG["T"]])
    t0 = time.perf_counter()
    g = orc.pinn_table(p, m)
    t_table = time.perf_counter() - t0
    # one bounded sample per step: the first Parareal iteration (F on all 32 slices,
    # correction, norm); a solve to 1e-6 with this coarse propagator needs at most P iterations
    t_iter = []
    for i in range(args.warmup + args.steps):
        s0 = time.perf_counter()
        orc.parareal(p, orc.COARSE_PINN, g=g, tol=0.0, max_iter=1)
        if i >= args.warmup:
            t_iter.append(time.perf_counter() - s0)
    it = statistics.mean(t_iter)
    K = CFG["P"]
    t_solve = t_table + K * it
    v = 1.0 / t_solve
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": it * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "coarse": "pinn"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", **host_cpu(),
                         "sample": f"per step one Parareal iteration over all {CFG['P']} slices; solve = network "
                                   f"table + {K} iterations (P, the count that reproduces serial fine)"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--train-steps", type=int, default=5000)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "fine", "batched", "large", "pinn", "train", "sweep", "generalize",
                             "datacoarse"],
                    help="fine / batched: only the fine propagator on all slices of the benchmark / "
                         "batched workload (profiling)")
    ap.add_argument("--batched", type=int, default=1, help="include the batched-workload leg (1/0)")
    ap.add_argument("--instances", type=int, default=4096, help="instances of --mode batched")
    ap.add_argument("--large-p", type=int, default=256, help="slices of --mode large")
    ap.add_argument("--large-steps", type=int, default=4096, help="CN steps per slice of --mode large")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.mode == "fine":
        run_fine_only(args)
    elif args.mode == "large":
        run_large(args)
    elif args.mode == "pinn":
        import torch

        from paper_2303_03848_b300 import binding as B
        from paper_2303_03848_b300 import build as BUILD

        BUILD.build()
        print(json.dumps(pinn_leg(B, torch)), flush=True)
    elif args.mode == "sweep":
        import torch

        from paper_2303_03848_b300 import binding as B
        from paper_2303_03848_b300 import build as BUILD

        BUILD.build()
        model, _ = train_network(B, torch, args.train_steps)
        print(json.dumps(sweep_leg(B, torch, model)), flush=True)
    elif args.mode == "generalize":
        import torch

        from paper_2303_03848_b300 import binding as B
        from paper_2303_03848_b300 import build as BUILD

        BUILD.build()
        print(json.dumps(generalize_leg(B, torch, args.train_steps)), flush=True)
    elif args.mode == "datacoarse":
        import torch

        from paper_2303_03848_b300 import binding as B
        from paper_2303_03848_b300 import build as BUILD

        BUILD.build()
        print(json.dumps(data_coarse_leg(B, torch, args.train_steps)), flush=True)
    elif args.mode == "train":
        import torch

        from paper_2303_03848_b300 import binding as B
        from paper_2303_03848_b300 import build as BUILD

        BUILD.build()
        print(json.dumps(train_leg(B, torch)), flush=True)
    elif args.mode == "batched":
        import torch

        from paper_2303_03848_b300 import binding as B
        from paper_2303_03848_b300 import build as BUILD

        BUILD.build()
        print(json.dumps(batched_leg(B, torch, n_inst=args.instances, solve=True, rule_too=True, pinn_solve=True)),
              flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
