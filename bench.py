#!/usr/bin/env python
"""Benchmark: diffraction patterns per second per ML-CG iteration on one GB300.

Workload: the production-size plain ML-CG problem -- 1024 x 1024 random-ellipse object,
128 x 128 Gaussian probe with quadratic phase, 60 x 60 jittered raster (3600 positions,
step 14, +-2 px), Poisson counts with peak 1e5 -- reconstructed from the uniform-ones
start.  A step is one CG iteration (GRAD, DIR, LS, Update of Algorithm 1).  The measured
data (236 MB) is larger than L2, so no flush is needed between steps.

Multi-GPU: the solve does not shard across GPUs; `--gpus N` (under torchrun) runs N
independent replicas and reports their total throughput (weak scaling).

`--impl reference` times the FP64 CPU oracle (the method's plain restatement) on the host
cores instead, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "diffraction patterns/s per CG iteration"
UNIT = "patterns/s"
WORKLOADS = {
    "production": "ml-cg 1024x1024 object, 128x128 probe, 3600 positions (60x60 raster, step 14, +-2), peak 1e5 counts",
    "spiral": "ml-cg 2048x2048 object, 256x256 probe, 10000 positions (Fermat spiral, +-2), peak 1e6 counts",
    "small": "ml-cg 256x256 object, 64x64 probe, 225 positions (15x15 raster, step 8, +-1), peak 1e4 counts",
    "gap": "ml-cg 1024x1024 object, 128x128 probe, 3600 positions (60x60 raster, step 14, +-2), peak 1e5 counts, "
           "test seed 5: time to relative objective gap 1e-3 per form",
    "views": "batched ml-cg: {n} views of 512^2-2048^2 (multiples of 128), 128x128 shared probe, rasters at 16 px "
             "(+-2), peak 1e5 counts, {k} positions in total",
}
WORKLOAD = WORKLOADS["production"]


def make_problem(name):
    from paper_2106_07575_gb300 import synth

    if name == "spiral":
        return synth.spiral_problem()
    if name == "small":
        return synth.small_problem()
    return synth.production_problem()


FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0

# DRAM traffic per launch of the LS pattern pass, from an ncu capture summarised in
# profiles/: valid only while the kernel's sources are the ones hashed there
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_ls_fft_mlcg_1024_p128.md")
TRAFFIC_SOURCES = ["fft_tile.cuh", "pattern_kernels.cuh", "pattern_p128.cu", "pty_internal.h", "reduce.cuh",
                   "mathx.cuh"]


def ls_pass_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_07575_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ls_pass_traffic(P, plan_ls):
    """(bytes per launch or None, note) for the chosen LS configuration (R, NT)."""
    import re

    try:
        with open(TRAFFIC_PROFILE) as fh:
            text = fh.read()
    except OSError:
        return None, "no profile summary"
    cur = ls_pass_source_hash()
    for m in re.finditer(r"^traffic: k_ls_fft<(\d+),(\d+),(\d+)> (\d+) bytes/launch, sources ([0-9a-f]+)$", text,
                         re.M):
        if (int(m.group(1)), int(m.group(2)), int(m.group(3))) != (P, plan_ls[0], plan_ls[1]):
            continue
        if m.group(5) != cur:
            return None, f"kernel sources changed since the capture ({m.group(5)} -> {cur})"
        return int(m.group(4)), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {os.path.basename(TRAFFIC_PROFILE)}"
    return None, f"no capture of k_ls_fft<{P},{plan_ls[0]},{plan_ls[1]}>"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pty", "reference"], default="pty")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ls-window", type=int, default=None)
    ap.add_argument("--tile-config", type=int, default=None)
    ap.add_argument("--workload", choices=["production", "spiral", "small", "views", "gap"], default="production")
    ap.add_argument("--pairs", type=int, default=200000, help="gap workload: training pairs of the learned start")
    ap.add_argument("--epochs", type=float, default=1.0, help="gap workload: passes over the training pairs")
    ap.add_argument("--views", type=int, default=64)
    ap.add_argument("--dft", type=int, default=0, help="0 FFT, 1 tensor-core split BF16, 2 split FP16")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 10]
        os.unlink(self.f.name)
        sm, smmax, reasons, busy = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                s, mx, util = float(r[1]), float(r[2]), float(r[4])
            except ValueError:
                continue
            smmax = mx
            sm.append(s)
            if util >= 50:
                busy.append(s)
            for n, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        use = busy or sm
        return {"sm_mhz": float(np.median(use)) if use else None, "sm_max_mhz": smmax,
                "reasons": sorted(reasons), "samples": len(rows), "samples_busy": len(busy)}


def fft2_flops(P):
    n = P * P
    return 5.0 * n * math.log2(n)


def over_ranks(dist, ms, units, device):
    """The job's time and work over all ranks (one process per GPU, each a replica of the
    path): the slowest rank's time and the sum of the ranks' units; every rank receives
    both.  dist None: one process, returned as given."""
    if dist is None:
        return ms, units
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args, rank):
    """FP64 CPU oracle on the host cores, one bounded sample of the workload per step."""
    if rank != 0:
        return
    import oracle
    from paper_2106_07575_gb300 import synth

    oracle.build()
    p = synth.production_problem()
    S = 400  # positions of the sample: the first 400 in raster order (a 1024^2 sub-scan)
    cores = os.cpu_count()
    pos, d = p.pos[:S], p.d[:S]
    psi = p.psi0()
    for _ in range(args.warmup):
        oracle.cg_solve(psi, p.probe, pos, d, 1, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.cg_solve(psi, p.probe, pos, d, 1, nthreads=cores)
    dt = time.perf_counter() - t0
    v = S * args.steps / dt
    sample = f"one FP64 oracle CG iteration over the first {S} of the 3600 positions per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_positions": S},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(p):
    import oracle

    oracle.build()
    cores = os.cpu_count()
    t0 = time.perf_counter()
    out = oracle.cg_solve(p.psi0(), p.probe, p.pos, p.d, 1, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": p.K / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one FP64 oracle CG iteration of the full workload ({p.K} positions, "
                      f"{int(out['halvings'][0])} line-search trials), {dt:.1f} s"}


def run_views(args, torch, pty, synth):
    """Batched form: every view of a series in one context (one launch per stage, graph replay)
    against the same views solved one after the other by single-view contexts."""
    probe, views = synth.view_batch(n_views=args.views, seed=3, P=128, step=16, jitter=2, peak=1e5, backend="torch")
    K = sum(len(pos) for _, pos, _ in views)
    stream = torch.cuda.current_stream()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pd = dev(probe)
    bctx = pty.BatchContext(pd, [(psi.shape[0], psi.shape[1], dev(pos), d) for psi, pos, d in views],
                            stream=stream.cuda_stream)
    psis = [torch.ones(psi.shape, dtype=torch.complex64, device="cuda") for psi, _, _ in views]
    bctx.cg_solve(psis, args.warmup)
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, reps = bctx.cg_solve(psis, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    plan = bctx.plan()
    bctx.close()
    done = sum(r["iters_done"] * len(v[1]) for r, v in zip(reps, views))
    # the same views, one single-view context after the other (creation not timed)
    seq_ms = 0.0
    seq_done = 0
    for psi, pos, d in views:
        ctx = pty.Context(pd, dev(pos), d, psi.shape[0], psi.shape[1], stream=stream.cuda_stream)
        x = torch.ones(psi.shape, dtype=torch.complex64, device="cuda")
        ctx.cg_solve(x, args.warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, r = ctx.cg_solve(x, args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        seq_ms += a.elapsed_time(b)
        seq_done += r["iters_done"] * len(pos)
        ctx.close()
    value = done / (ms * 1e-3)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["views"].format(n=len(views), k=K), "plan": plan,
                   "l2": "inputs larger than L2"},
        "status": pty.STATUS_NAMES[st], "clocks": clocks,
        "sequential": {"value": seq_done / (seq_ms * 1e-3), "ms_total": seq_ms,
                       "note": "the same views solved one after the other by single-view contexts"},
        "speedup_vs_sequential": (done / ms) / (seq_done / seq_ms),
    }), flush=True)


def run_gap(args, torch, pty, synth):
    """Wall time to a relative objective gap of 1e-3 (gap_m = (F_m - F*) / (F_0^ones - F*),
    F* = F(psi_true)) on the learned-init test geometry, per form: plain FP32 FFT from the
    ones start, split-BF16 and split-FP16 tensor-core DFTs from the ones start, and the
    learned start (network trained here on forward-model pairs; training time reported
    apart, prediction + stitching + both start objectives counted with the solve)."""
    from paper_2106_07575_gb300 import learned

    prob = synth.production_problem(seed=5)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    probe, pos, d = dev(prob.probe), dev(prob.pos), dev(prob.d)
    psi_true = dev(prob.psi_true)
    cap = 4 * prob.niter
    forms = {}
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()

    def solve_from(ctx, start):
        ctx.cg_reset()
        x = start.clone()
        ctx.cg_solve(x.clone(), 2)  # warm the captured iteration
        ctx.cg_reset()
        it, ms, F = learned.solve_to_gap(ctx, x, F_star, F0, cap, chunk=1)
        return it, ms, F

    base = pty.Context(probe, pos, d, prob.H, prob.W)
    g = torch.empty_like(psi_true)
    F_star = base.gradient(psi_true, g)
    ones = torch.ones_like(psi_true)
    F0 = base.gradient(ones, g)
    for name, dft in (("plain FP32 FFT, ones start", 0), ("split BF16 tensor-core DFT, ones start", 1),
                      ("split FP16 tensor-core DFT, ones start", 2)):
        opts = pty.default_opts()
        opts.dft = dft
        ctx = base if dft == 0 else pty.Context(probe, pos, d, prob.H, prob.W, opts)
        it, ms, F = solve_from(ctx, ones)
        forms[name] = {"iterations": it, "ms": ms if it is not None else None,
                       "ms_per_iteration": ms / max(len(F) - 1, 1)}
        if ctx is not base:
            ctx.close()
    # learned start
    t0 = time.perf_counter()
    d_tr, t_tr = learned.training_pairs(prob.probe, args.pairs)
    gen_s = time.perf_counter() - t0
    net = pty.Network(prob.P, 32, 6, max_batch=64)
    net.init_params(7)
    net.set_loss_weight((np.abs(prob.probe.astype(np.complex128)) ** 2).astype(np.float32))
    steps = max(1, int(round(args.epochs * args.pairs / 64)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train(d_tr, t_tr, 64, steps, seed=9)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del d_tr, t_tr
    psi0 = torch.empty_like(psi_true)
    net.learned_init(base, d, psi0)  # warm
    rep = net.learned_init(base, d, psi0)
    it, ms, F = solve_from(base, psi0)
    conv_flop = 2 * prob.P * prob.P * (9 * 32 + 4 * 9 * 32 * 32 + 9 * 32 * 2)  # one image, forward
    forms["learned start (CNN + stitch), FP32 FFT"] = {
        "iterations": it, "ms": (ms + rep["ms"]) if it is not None else None, "ms_init": rep["ms"],
        "used_learned": rep["used_learned"], "scale": rep["scale"],
        "gap_at_start": (min(rep["F_learned"], rep["F_ones"]) - F_star) / (F0 - F_star),
        "gap_learned_start": (rep["F_learned"] - F_star) / (F0 - F_star),
        "training": {"pairs": args.pairs, "steps": steps, "batch": 64, "generate_s": gen_s, "train_s": train_s,
                     "pairs_per_s": steps * 64 / train_s,
                     "conv_tflops": 3 * conv_flop * steps * 64 / train_s / 1e12,
                     "loss_first": float(losses[:16].mean()), "loss_last": float(losses[-100:].mean())}}
    clocks = clk.stop()
    base.close()
    plain = forms["plain FP32 FFT, ones start"]
    print(json.dumps({
        "metric": "wall time to relative objective gap 1e-3", "value": plain["ms"], "unit": "ms", "n_gpus": 1,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["gap"], "cap_iterations": cap, "F_star": F_star, "F0_ones": F0},
        "forms": forms, "clocks": clocks}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    from paper_2106_07575_gb300 import pty, synth

    torch.cuda.set_device(local)
    if args.workload == "views":
        run_views(args, torch, pty, synth)
        return
    if args.workload == "gap":
        run_gap(args, torch, pty, synth)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    p = make_problem(args.workload)
    workload = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    opts = pty.default_opts()  # the defaults: one CG iteration replayed as a CUDA graph
    if args.ls_window:
        opts.ls_window = args.ls_window
    if args.tile_config is not None:
        opts.tile_config = args.tile_config
    opts.dft = args.dft
    probe_d, pos_d, d_d = dev(p.probe), dev(p.pos), dev(p.d)
    ctx = pty.Context(probe_d, pos_d, d_d, p.H, p.W, opts, stream=stream.cuda_stream)
    psi = dev(p.psi0())
    ctx.cg_solve(psi, args.warmup)

    clk = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    st, rep = ctx.cg_solve(psi, args.steps)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist:
        dist.barrier()
    steps_done = rep["iters_done"]
    ms, units = over_ranks(dist, t_start.elapsed_time(t_end), p.K * steps_done, "cuda")
    plan = ctx.plan()
    ctx.close()

    # per-kernel launch durations: the same workload in a second context with per-stage
    # CUDA events on the stream the kernels run on (no graph replay there); 1 warm-up and up
    # to 10 iterations continuing from the timed solve's object
    topts = pty.default_opts()
    topts.ls_window, topts.tile_config, topts.dft, topts.flags = opts.ls_window, opts.tile_config, opts.dft, 1
    tctx = pty.Context(probe_d, pos_d, d_d, p.H, p.W, topts, stream=stream.cuda_stream)
    tctx.cg_solve(psi, 1)
    tctx.stage_times(reset=True)
    n_stage = max(1, min(args.steps, 10))
    _, trep = tctx.cg_solve(psi, n_stage)
    stage_ms, stage_n = tctx.stage_times(reset=True)
    tctx.close()
    n_it = max(trep["iters_done"], 1)

    # roofline of the LS pattern pass k_ls_fft, one of the two largest kernels with the linear
    # GRAD pass (whose time and rate go to "other"), and the one with a current traffic
    # capture (FP32 ALU bound: one 2-D FFT per pattern on the CUDA cores; one launch per
    # iteration covers all K patterns).
    # Algorithmic flops: 5 N log2 N per 2-D DFT (N = P^2) plus the probe product (6 N) and,
    # at the n_e detector pixels with counts, the two Parseval sums (8 per pixel).
    P, K = p.P, p.K
    L = opts.ls_window
    n_e = float(np.count_nonzero(p.d))  # detector pixels with counts
    ls_flops = K * (fft2_flops(P) + 6 * P * P) + 8 * n_e
    ls_ms = stage_ms[2] / max(stage_n[2], 1)
    grad_ms = stage_ms[0] / max(stage_n[0], 1)
    peak_tflops = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = ls_flops / (ls_ms * 1e-3) / 1e12
    traffic, traffic_note = ls_pass_traffic(P, plan["ls"])
    roof = {"bound": "alu", "kernel": "k_ls_fft", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": traffic, "traffic_note": traffic_note,
            "peak_note": "FP32 FMA peak derived: 152 SMs x 128 lanes x 2 flop x 2070 MHz",
            "launch_ms": ls_ms, "launches_timed": int(stage_n[2]),
            "timing": "CUDA events around each k_ls_fft launch on its stream, stage-timed pass of the same workload",
            "other": {"grad_pass_ms": grad_ms,
                      "grad_pass_tflops_linear_form": K * (fft2_flops(P) + 6 * P * P) / (grad_ms * 1e-3) / 1e12,
                      "ls_windows_ms_per_iter": stage_ms[4] / n_it, "scatter_ms_per_iter": stage_ms[1] / n_it,
                      "small_ms_per_iter": stage_ms[3] / n_it}}

    Lcap = 32 if L == 0 else L
    first_w = 4 if L == 0 else L
    nwin = 1 + (max(0, opts.max_halvings - first_w) + Lcap - 1) // Lcap
    # per iteration: grad (full and linear form, one returns at once), scatter, dy_finalize,
    # eta, LS pass, windows (entries + decide; the adaptive first window launches the 8-, 16-
    # and 32-candidate entry kernels, all but one returning at once, after the certificate
    # kernel), update + counters; per call: 2 hashes, hash check, begin, hash store
    launches = args.steps * (8 + 2 * nwin + (3 if L == 0 else 0)) + 5 if args.dft == 0 else None
    value = units / (ms * 1e-3)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / max(steps_done, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "ls_window": L, "tile_config": opts.tile_config, "plan": plan,
                   "dft": ["fp32 fft", "tensor-core split bf16", "tensor-core split fp16"][args.dft],
                   "l2": f"inputs larger than L2 ({p.d.nbytes / 1e6:.0f} MB data)",
                   "parallelism": f"{world} independent replica(s)"},
        "status": pty.STATUS_NAMES[st], "roofline": roof, "clocks": clocks, "gpu_launches": launches,
        "stages_ms_per_iter": {"grad": stage_ms[0] / n_it, "scatter": stage_ms[1] / n_it,
                               "ls_pass": stage_ms[2] / n_it, "ls_windows": stage_ms[4] / n_it,
                               "small": stage_ms[3] / n_it, "iterations": n_it,
                               "note": "stage-timed pass (events between stages, no graph)"},
        "trials_per_iter": float(np.mean(rep["halvings"])) if len(rep["halvings"]) else None,
    }

    if not args.no_e2e:
        # end to end through the C ABI with pinned host buffers: create (copies data) + K
        # single-iteration solves (psi in and out every step) + destroy
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        d_h, psi_h, probe_h, pos_h = pin(p.d), pin(p.psi0()), pin(p.probe), pin(p.pos)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        ctx2 = pty.Context(probe_h, pos_h, d_h, p.H, p.W, None, stream=stream.cuda_stream)
        for _ in range(args.steps):
            ctx2.cg_solve(psi_h, 1)
        ctx2.close()
        e2e_s, e2e_units = over_ranks(dist, time.perf_counter() - t0, K * args.steps, "cuda")
        once = d_h.nbytes + probe_h.nbytes + pos_h.nbytes
        out["e2e"] = {"value": e2e_units / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": int(psi_h.nbytes + once / args.steps),
                      "d2h_bytes_per_step": int(psi_h.nbytes + 8 * 4 + 4),
                      "note": "pty_create from host arrays + one pty_cg_solve(niter=1) per step with host psi"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "production":
        out["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
