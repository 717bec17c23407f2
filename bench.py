#!/usr/bin/env python
"""Benchmark: diffraction patterns per second per ML-CG iteration on one GB300.

Workload: the production-size plain ML-CG problem -- 1024 x 1024 random-ellipse object,
128 x 128 Gaussian probe with quadratic phase, 60 x 60 jittered raster (3600 positions,
step 14, +-2 px), Poisson counts with peak 1e5 -- reconstructed from the uniform-ones
start.  A step is one CG iteration (GRAD, DIR, LS, Update of Algorithm 1).  The measured
data (236 MB) is larger than L2, so no flush is needed between steps.

Multi-GPU: the solve does not shard across GPUs; `--gpus N` (under torchrun) runs N
independent replicas and reports their total throughput (weak scaling).

Timed region: after W warm-up iterations the CG state is checkpointed; the K-step solve is
replayed from that checkpoint for about a second (so that the clock sampler sees the GPU
under load), then restored once more and the K steps are timed with CUDA events: the
timed steps are iterations W .. W+K-1 of one solve.

`--impl reference` times the FP64 CPU oracle (the method's plain restatement) on the host
cores instead: the same workload, the same iterations W .. W+K-1 of a solve from the same
start (bounded to a few minutes of CPU time).
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
    "subpixel": "ml-cg 1024x1024 object, 128x128 probe, 3600 sub-pixel positions (60x60 raster, step 14, uniform "
                "real jitter +-2, one Fourier-shifted probe per position), peak 1e5 counts",
    "gap": "ml-cg 1024x1024 object, 128x128 probe, 3600 positions (60x60 raster, step 14, +-2), peak 1e5 counts, "
           "test seed 5: time to relative objective gap 1e-3 per form",
    "spiral_gap": "ml-cg 2048x2048 object, 256x256 probe, 10000 positions (Fermat spiral, +-2), peak 1e6 counts: "
                  "time to relative objective gap 1e-3 from the ones start, FP32 FFT and split-BF16 tensor-core DFT",
    "train": "learned start: 6-layer 3x3 CNN (1-32-32-32-32-32-2 channels), 128x128 patterns, batch 64, "
             "2048 forward-model pairs (Poisson counts of |F[p psi]|^2 of ellipse phantoms, peak 1e5 probe)",
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
    if name == "subpixel":
        return synth.subpixel_problem(H=1024, W=1024, P=128, n=60, step=14, jitter=2.0, peak=1e5, seed=1, niter=64)
    return synth.production_problem()


FP32_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0

# DRAM traffic per launch of a pattern kernel, from the one-pass ncu captures summarised in
# profiles/: valid only while the kernel's sources are the ones hashed there
TRAFFIC_PROFILES = {"k_ls_fft": os.path.join(ROOT, "profiles", "k_ls_fft_mlcg_1024_p128.md"),
                    "k_grad_lin": os.path.join(ROOT, "profiles", "k_grad_lin_mlcg_1024_p128.md")}
TRAFFIC_SOURCES = ["fft_tile.cuh", "pattern_kernels.cuh", "pattern_p128.cu", "pty_internal.h", "reduce.cuh",
                   "mathx.cuh"]


def pattern_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_07575_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel, P, plan):
    """(bytes per launch or None, note) of `kernel` in the configuration (R, NT) = plan."""
    import re

    path = TRAFFIC_PROFILES[kernel]
    try:
        with open(path) as fh:
            text = fh.read()
    except OSError:
        return None, "no profile summary"
    cur = pattern_source_hash()
    pat = r"^traffic: " + kernel + r"<(\d+),(\d+),(\d+)> (\d+) bytes/launch, sources ([0-9a-f]+)$"
    for m in re.finditer(pat, text, re.M):
        if (int(m.group(1)), int(m.group(2)), int(m.group(3))) != (P, plan[0], plan[1]):
            continue
        if m.group(5) != cur:
            return None, f"kernel sources changed since the capture ({m.group(5)} -> {cur})"
        return int(m.group(4)), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {os.path.basename(path)}"
    return None, f"no capture of {kernel}<{P},{plan[0]},{plan[1]}>"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--preroll-s", type=float, default=1.0,
                    help="seconds of replayed steps before the timed steps (clock sampling under load)")
    ap.add_argument("--impl", choices=["pty", "reference"], default="pty")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ls-window", type=int, default=None)
    ap.add_argument("--tile-config", type=int, default=None)
    ap.add_argument("--workload", choices=["production", "spiral", "small", "subpixel", "views", "gap", "spiral_gap",
                                           "train"],
                    default="production")
    ap.add_argument("--pairs", type=int, default=200000, help="gap workload: training pairs of the learned start")
    ap.add_argument("--epochs", type=float, default=1.0, help="gap workload: passes over the training pairs")
    ap.add_argument("--views", type=int, default=64)
    ap.add_argument("--dft", type=int, default=0, help="0 FFT, 1 tensor-core split BF16, 2 split FP16")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling (every 20 ms) around the timed region.  Samples carry their
    timestamps; the record reports the samples taken while the GPU ran the replayed steps
    and the timed steps (`window`), and how many fell inside the timed steps alone."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
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

    def stop(self, load=None, timed=None):
        """load, timed: (t0, t1) wall-clock windows (time.time()) of the GPU work."""
        import datetime

        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 11]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm_all, sm_load, n_timed, smmax, reasons, power = [], [], 0, None, set(), []
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                s, mx, pw = float(r[2]), float(r[3]), float(r[4])
            except ValueError:
                continue
            smmax = mx
            sm_all.append(s)
            in_load = load is not None and load[0] <= ts <= load[1]
            if in_load:
                sm_load.append(s)
                power.append(pw)
                for n, v in zip(names, r[7:11]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            if timed is not None and timed[0] <= ts <= timed[1]:
                n_timed += 1
        use = sm_load or sm_all
        return {"sm_mhz": float(np.median(use)) if use else None, "sm_max_mhz": smmax,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(sm_load),
                "samples_in_timed_steps": n_timed,
                "power_w_median": float(np.median(power)) if power else None,
                "window": "samples taken while the replayed and the timed steps ran" if sm_load else
                          "no sample fell under load: median of all samples"}


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


REF_MAX_ITERS = 80  # bound of the oracle's solve (about 2 minutes on 16 host cores)


def oracle_rate(p, warmup, steps, cores):
    """The FP64 oracle's throughput on iterations warmup .. warmup+k-1 of one solve of the
    workload from its start (the iterations the GPU arm times), k <= steps bounded so the
    solve stays within REF_MAX_ITERS iterations.  Returns (patterns/s, k, seconds, trials)."""
    import oracle

    oracle.build()
    k = max(1, min(steps, REF_MAX_ITERS - warmup))
    out = oracle.cg_solve(p.psi0(), p.probe, p.pos, p.d, warmup + k, nthreads=cores)
    t = out["t"]
    done = len(t) - warmup
    if done < 1:
        raise RuntimeError(f"oracle solve stopped after {len(t)} iterations (status {out['status']})")
    k = min(k, done)
    t0 = t[warmup - 1] if warmup >= 1 else 0.0
    dt = float(t[warmup + k - 1] - t0)
    trials = out["halvings"][warmup:warmup + k]
    return p.K * k / dt, k, dt, float(np.mean(trials))


def run_reference(args, rank):
    """FP64 CPU oracle on the host cores: the GPU arm's workload and timed iterations."""
    if rank != 0:
        return
    from paper_2106_07575_gb300 import synth

    p = synth.production_problem()
    cores = os.cpu_count()
    v, k, dt, trials = oracle_rate(p, args.warmup, args.steps, cores)
    sample = (f"iterations {args.warmup}..{args.warmup + k - 1} of one FP64 oracle ML-CG solve of the full workload "
              f"({p.K} positions, {trials:.1f} line-search trials per iteration) from the ones start, "
              f"{dt:.1f} s timed; the {args.warmup} earlier iterations untimed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": k, "warmup": args.warmup, "ms_per_step": 1e3 * dt / k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "timed_iterations": [args.warmup, args.warmup + k - 1]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def oracle_single_thread(p):
    """The oracle on one host core: the first iteration of a solve of the full workload."""
    import oracle

    oracle.build()
    out = oracle.cg_solve(p.psi0(), p.probe, p.pos, p.d, 1, nthreads=1)
    dt = float(out["t"][0])
    return {"value": p.K / dt, "unit": UNIT, "cores": 1,
            "sample": f"iteration 0 of one single-threaded FP64 oracle solve of the full workload "
                      f"({p.K} positions, {int(out['halvings'][0])} line-search trials), {dt:.1f} s"}


def cpu_baseline(p, warmup):
    """The oracle on a bounded sample of the GPU arm's timed iterations (about 10-20 s) on all
    host cores, and on one core for the solve's first iteration."""
    cores = os.cpu_count()
    v, k, dt, trials = oracle_rate(p, warmup, 5, cores)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"iterations {warmup}..{warmup + k - 1} of one FP64 oracle solve of the full workload "
                      f"({p.K} positions, {trials:.1f} line-search trials per iteration), {dt:.1f} s timed",
            "single_thread": oracle_single_thread(p)}


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


def run_spiral_gap(args, torch, pty, synth):
    """Wall time and iterations to a relative objective gap of 1e-3 (gap_m = (F_m - F*) /
    (F_0 - F*), F* = F(psi_true), F_0 = F(ones)) on the spiral workload (P = 256) from the
    ones start, for the FP32 FFT and the split-BF16 tensor-core DFT; one host read of the
    objective per iteration in both."""
    from paper_2106_07575_gb300 import learned

    prob = synth.spiral_problem()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    probe, pos, d = dev(prob.probe), dev(prob.pos), dev(prob.d)
    psi_true = dev(prob.psi_true)
    cap = 300  # the spiral workload states no iteration count; the production one needs 64
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    base = pty.Context(probe, pos, d, prob.H, prob.W)
    g = torch.empty_like(psi_true)
    F_star = base.gradient(psi_true, g)
    ones = torch.ones_like(psi_true)
    F0 = base.gradient(ones, g)
    forms = {}
    clk.start()
    t_load0 = time.time()
    for name, dft in (("plain FP32 FFT", 0), ("split BF16 tensor-core DFT", 1)):
        opts = pty.default_opts()
        opts.dft = dft
        ctx = base if dft == 0 else pty.Context(probe, pos, d, prob.H, prob.W, opts)
        ctx.cg_solve(ones.clone(), 2)  # warm the captured iteration
        ctx.cg_reset()
        x = ones.clone()
        it, ms, F = learned.solve_to_gap(ctx, x, F_star, F0, cap, chunk=1)
        forms[name] = {"iterations": it, "ms": ms if it is not None else None,
                       "ms_per_iteration": ms / max(len(F) - 1, 1), "final_gap": (F[-1] - F_star) / (F0 - F_star)}
        if ctx is not base:
            ctx.close()
    clocks = clk.stop(load=(t_load0, time.time()))
    base.close()
    plain = forms["plain FP32 FFT"]
    print(json.dumps({
        "metric": "wall time to relative objective gap 1e-3", "value": plain["ms"], "unit": "ms", "n_gpus": 1,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["spiral_gap"], "cap_iterations": cap, "F_star": F_star, "F0_ones": F0},
        "forms": forms, "clocks": clocks}), flush=True)


def run_train(args, torch, pty, synth):
    """CNN training throughput (pairs/s) of the learned start through pty_cnn_train: K steps of
    batch 64 (forward, loss, backward, Adam) timed with CUDA events on the library's stream
    after W warm-up steps; hidden layers on the tensor cores, and the same steps with them
    switched off for comparison."""
    from paper_2106_07575_gb300 import learned

    prob = synth.production_problem(seed=5)
    n_pairs, B, L = 2048, 64, 6
    d_tr, t_tr = learned.training_pairs(prob.probe, n_pairs, per_phantom=n_pairs, phantoms=("ellipse",))
    stream = torch.cuda.current_stream()
    net = pty.Network(prob.P, 32, L, max_batch=B, stream=stream.cuda_stream)
    net.init_params(7)
    net.set_loss_weight((np.abs(prob.probe.astype(np.complex128)) ** 2).astype(np.float32))
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    rates = {}
    for name, tc in (("cuda cores", 0), ("tensor cores", 1)):
        prev = pty.pty_selftest_cnn_tc(tc)
        net.train(d_tr, t_tr, B, max(args.warmup, 3), seed=1)
        torch.cuda.synchronize()
        if tc:  # clocks sampled over preroll steps (args.preroll_s seconds) and the timed steps
            clk.start()
            t_load0 = time.time()
            while time.time() - t_load0 < args.preroll_s:
                net.train(d_tr, t_tr, B, 20, seed=3)
                torch.cuda.synchronize()
        tw0 = time.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        losses = net.train(d_tr, t_tr, B, args.steps, seed=2)
        e1.record(stream)
        torch.cuda.synchronize()
        if tc:
            clocks = clk.stop(load=(t_load0, time.time()), timed=(tw0, time.time()))
        pty.pty_selftest_cnn_tc(prev)
        ms = e0.elapsed_time(e1)
        rates[name] = {"pairs_per_s": args.steps * B / (ms / 1e3), "ms_per_step": ms / args.steps,
                       "loss_last": float(losses[-1])}
    tcr = rates["tensor cores"]
    print(json.dumps({
        "metric": "CNN training pairs per second", "value": tcr["pairs_per_s"], "unit": "pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": tcr["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (split bf16 tensor cores)",
        "data": "synthetic", "config": {"workload": WORKLOADS["train"], "l2": "inputs larger than L2 per step"},
        "forms": rates, "gpu_launches": (5 * L + 3) * args.steps, "clocks": clocks}), flush=True)


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
    if args.workload == "train":
        run_train(args, torch, pty, synth)
        return
    if args.workload == "spiral_gap":
        run_spiral_gap(args, torch, pty, synth)
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
    if args.warmup > 0:
        ctx.cg_solve(psi, args.warmup)
    # checkpoint after the warm-up: every replay below and the timed steps start here
    ckpt = ctx.state_save()
    psi_ck = psi.clone()

    def restore():
        ctx.state_load(ckpt)
        psi.copy_(psi_ck)

    clk = Clocks(local)
    clk.start()
    time.sleep(0.1)
    torch.cuda.synchronize()
    t_load0 = time.time()
    while True:  # replay the timed solve so the sampler sees the GPU under load
        restore()
        ctx.cg_solve(psi, args.steps)
        torch.cuda.synchronize()
        if time.time() - t_load0 >= args.preroll_s:
            break
    restore()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    t_start.record(stream)
    st, rep = ctx.cg_solve(psi, args.steps)
    t_end.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    time.sleep(0.05)
    clocks = clk.stop(load=(t_load0, tw1), timed=(tw0, tw1))
    steps_done = rep["iters_done"]
    ms, units = over_ranks(dist, t_start.elapsed_time(t_end), p.K * steps_done, "cuda")
    plan = ctx.plan()

    # Per-kernel launch durations: the same iterations in a second context with CUDA events
    # around each stage on the stream the kernels run on (no graph there).  The GRAD stage
    # launches both GRAD kernels (the full form on a call's first iteration, the linear form
    # after it; the other returns at once), so the linear form's time is the difference of a
    # one-iteration and an n-iteration call from the same checkpoint, over n - 1.
    topts = pty.default_opts()
    topts.ls_window, topts.tile_config, topts.dft, topts.flags = opts.ls_window, opts.tile_config, opts.dft, 1
    tctx = pty.Context(probe_d, pos_d, d_d, p.H, p.W, topts, stream=stream.cuda_stream)
    n_stage = max(2, min(args.steps, 21))

    def staged(n):
        tctx.state_load(ckpt)
        x = psi_ck.clone()
        tctx.cg_solve(x, 1)  # warm the kernels of this context
        tctx.state_load(ckpt)
        x.copy_(psi_ck)
        tctx.stage_times(reset=True)
        _, r = tctx.cg_solve(x, n)
        ms_, n_ = tctx.stage_times(reset=True)
        return ms_, n_, max(r["iters_done"], 1)

    s1_ms, _, _ = staged(1)
    stage_ms, stage_n, n_it = staged(n_stage)
    tctx.close()
    ctx.close()

    P, K = p.P, p.K
    L = opts.ls_window
    n_e = float(np.count_nonzero(p.d))  # detector pixels with counts
    # Algorithmic flops per launch (all K patterns): one 2-D FFT per pattern at 5 N log2 N
    # (N = P^2) plus the probe product (6 N); at the n_e pixels with counts the LS pass forms
    # two Parseval sums and two certificate sums (8 + 6 per pixel), the linear GRAD pass
    # updates u, forms the residual correction and the log term (about 20 per pixel).
    fft_part = K * (fft2_flops(P) + 6 * P * P)
    kern = {"k_grad_lin": {"flops": fft_part + 20 * n_e, "plan": plan["grad"],
                           "ms": (stage_ms[0] - s1_ms[0]) / max(n_it - 1, 1),
                           "timing": "GRAD stage of an n-iteration call minus that of a 1-iteration call "
                                     "from the same checkpoint, over n - 1 (CUDA events on the library's stream)"},
            "k_ls_fft": {"flops": fft_part + 14 * n_e, "plan": plan["ls"], "ms": stage_ms[2] / max(stage_n[2], 1),
                         "timing": "CUDA events around each k_ls_fft launch on the library's stream"}}
    dom = max(kern, key=lambda k: kern[k]["ms"])
    peak_max = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    sm_mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    peak_sampled = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12

    def roof_of(name):
        k = kern[name]
        ach = k["flops"] / (k["ms"] * 1e-3) / 1e12
        traffic, note = kernel_traffic(name, P, k["plan"])
        return {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak_max, "unit": "TFLOP/s",
                "frac": ach / peak_max, "traffic": traffic, "traffic_note": note,
                "peak_note": "FP32 FMA peak derived (of derived, no FP32 figure in the measured peaks): "
                             f"152 SMs x 128 lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz (maximum SM clock)",
                "peak_at_sampled_clock": peak_sampled, "frac_at_sampled_clock": ach / peak_sampled,
                "sampled_sm_mhz": sm_mhz, "launch_ms": k["ms"], "flops_per_launch": k["flops"],
                "timing": k["timing"]}

    roof = roof_of(dom)
    other = [n for n in kern if n != dom][0]
    roof["other"] = {other: {kk: roof_of(other)[kk] for kk in ("achieved", "frac", "launch_ms", "traffic")},
                     "scatter_ms_per_iter": stage_ms[1] / n_it, "ls_windows_ms_per_iter": stage_ms[4] / n_it,
                     "small_ms_per_iter": stage_ms[3] / n_it}

    Lcap = 32 if L == 0 else L
    first_w = 4 if L == 0 else L
    nwin = 1 + (max(0, opts.max_halvings - first_w) + Lcap - 1) // Lcap
    # per iteration: grad (full and linear form, one returns at once), scatter, dy_finalize,
    # eta, LS pass, windows (entries + decide; the adaptive first window launches the 6-, 8-,
    # 16- and 32-candidate entry kernels, all but one returning at once, after the certificate
    # kernel), update + counters; per call: 2 hashes, hash check, begin, hash store
    launches = args.steps * (8 + 2 * nwin + (4 if L == 0 else 0)) + 5 if args.dft == 0 else None
    value = units / (ms * 1e-3)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / max(steps_done, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "ls_window": L, "tile_config": opts.tile_config, "plan": plan,
                   "dft": ["fp32 fft", "tensor-core split bf16", "tensor-core split fp16"][args.dft],
                   "l2": f"inputs larger than L2 ({p.d.nbytes / 1e6:.0f} MB data)",
                   "timed_iterations": [args.warmup, args.warmup + steps_done - 1],
                   "parallelism": f"{world} independent replica(s)"},
        "status": pty.STATUS_NAMES[st], "roofline": roof, "clocks": clocks, "gpu_launches": launches,
        "stages_ms_per_iter": {"grad": stage_ms[0] / n_it, "scatter": stage_ms[1] / n_it,
                               "ls_pass": stage_ms[2] / n_it, "ls_windows": stage_ms[4] / n_it,
                               "small": stage_ms[3] / n_it, "iterations": n_it,
                               "note": "stage-timed call from the checkpoint (events between stages, no graph)"},
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
        out["cpu_baseline"] = cpu_baseline(p, args.warmup)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
