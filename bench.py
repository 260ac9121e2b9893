#!/usr/bin/env python3
"""Benchmark: seconds per reconstruction iteration (Algorithm 2 step: NPC, forward, FP64 loss,
adjoint, Adam) on the paper's in-vivo scale -- 256 x 256 x 128 = 8.4 M Gaussians on a 0.1 mm
grid, 1024 sensors, 4096 samples at 40 MHz -- with seeded synthetic data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  `value` is device time per iteration with inputs resident in
HBM; `e2e` repeats the measurement through the public API with the measured signal copied from
pinned host memory each step and the loss read back.  `roofline` uses the dominant kernel's own
launch times (CUDA events on its stream, inside the timed region): the direct windowed
evaluation's FP32 and MUFU work over that time, against the slower pipe's issue rate.
`cpu_baseline` times the FP64 oracle on a bounded sensor sample (rank 0, N = 1 only).
With N > 1 (torchrun) every rank runs an independent replica (the path is replicated, not
sharded, on one-GPU machines): value = max-over-ranks time / (K * N).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per IR iteration (fwd+adjoint) at 8.4M Gaussians; pair-evals/s vs FP32 peak"
UNIT = "s/iter"
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
MUFU_LANES_PER_SM = 32          # MUFU lanes per SM (ex2 measured at ~30 lane-ops / clk / SM)
LAUNCHES_PER_STEP = 10          # npc, slab info, forward, slab reduce, resid, finish, Q table, adjoint, schedule, adam
ASSA_NMIN = 25                  # the paper's minimum number of fine samples across the pulse


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0               # the recipe's fallback


HBM_GBS = _measured_hbm()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="paper", choices=["paper", "mid", "tiny"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sensors", type=int, default=32)
    p.add_argument("--no-assa", action="store_true",
                   help="skip timing the paper's ASSA operator, the regulariser, voxelization, the image metrics "
                        "and the differentiation workload")
    p.add_argument("--no-warmstart", action="store_true", help="skip the learned warm-start comparison (~3 min)")
    p.add_argument("--ws-train", type=int, default=2000)
    p.add_argument("--ws-eval", type=int, default=200)
    p.add_argument("--ws-epochs", type=int, default=1)
    return p.parse_args()


def workload(name):
    from paper_2602_03893_gb300 import synth
    return {"paper": synth.paper_scale, "mid": synth.mid, "tiny": synth.tiny}[name]()


def pairs_of(w):
    return float(w.M) * w.Nd


def work_units(w):
    """pair-evals and sample-evals per operator application.  Every pair's window lies inside
    the record for these workloads; the expected number of samples in |d| <= k sigma is
    2 k sigma / (v / fs) (an interval of that length in sample units)."""
    pairs = float(w.M) * w.Nd
    samples = pairs * 2.0 * w.k * w.grid.sigma * w.fs / w.v
    return pairs, samples


# Algorithmic work of the direct windowed evaluation (the operator's definition): per sample-eval
# 1 exponential (MUFU) and 4 FP32 ops (form d, scale d^2, d * A / 2R, accumulate; the adjoint adds
# 1 FMA with delta); per pair 10 FP32 ops (offset distance, phase, window bounds, weight) and 2 MUFU
# ops (rsqrt, rcp).  The bound is the slower pipe: T = max(F / P_fp32, X / P_mufu).  The kernels
# factor the sample loop through sub-sample moments and execute fewer operations than this; the
# fraction is the direct evaluation's work over the measured time.
FP32_PER_SAMPLE = {"forward": 4.0, "adjoint": 5.0}
FP32_PER_PAIR = 10.0
MUFU_PER_SAMPLE = 1.0
MUFU_PER_PAIR = 2.0
# The full gradient (amplitude, centre, width) of the direct windowed evaluation: per sample-eval
# the phase, the exponential and four accumulated moments of delta e (delta e d^0..3): 10 FP32
# ops and 1 MUFU; per pair the phase and weight (10 FP32, 2 MUFU) plus the gradient assembly
# (dp/dR, the three centre components, dp/dsigma, and their sums over sensors: 30 FP32, 2 MUFU).
FULL_FP32_PER_SAMPLE, FULL_FP32_PER_PAIR = 10.0, 40.0
FULL_MUFU_PER_SAMPLE, FULL_MUFU_PER_PAIR = 1.0, 4.0


def alg_work(w, op):
    """(FP32 lane-ops, MUFU lane-ops) of one operator application."""
    pairs, samples = work_units(w)
    return (FP32_PER_SAMPLE[op] * samples + FP32_PER_PAIR * pairs,
            MUFU_PER_SAMPLE * samples + MUFU_PER_PAIR * pairs)


def kernel_names(w):
    """Kernels the library launches for the two operators on this workload: the moment kernels
    when the grid's shared sigma admits the sub-sample expansion (Delta <= sigma / 2)."""
    if w.v / w.fs <= 0.5 * w.grid.sigma:
        return {"forward": "fwd_lanes_kernel", "adjoint": "adj_moment_kernel"}
    return {"forward": "fwd_grid_kernel", "adjoint": "adj_kernel"}


def diff_leg(args, dev, stream, p_fp32, p_mufu, pipe_peaks, world):
    """The differentiation workload: 262,144 free Gaussians (64^3 lattice jittered by U[+-0.05] mm,
    sigma log-uniform 0.05-0.2 mm), 512 sensors x 2048 samples.  Amplitudes dense (U[0,1]^2, as
    an optimisation iterate has them).  Times gpair_forward (free centres: tile and slab summaries,
    fwd_free_lanes_kernel, slab reduction) and gpair_adjoint with all three gradients (tile summaries,
    adj_kernel with the centre and width derivatives) on the stream, CUDA events, after warm-up."""
    import torch

    from paper_2602_03893_gb300 import _lib, synth
    w = synth.differentiable(4)
    cx, cy, cz, sg, _ = w.free
    rng = np.random.default_rng(9)
    A = (rng.uniform(0.0, 1.0, w.M) ** 2).astype(np.float32)
    t = lambda q: torch.as_tensor(np.ascontiguousarray(q, dtype=np.float32), device=dev)
    gs = _lib.Gaussians(A=t(A), cx=t(cx), cy=t(cy), cz=t(cz), sigma=t(sg))
    arr = _lib.SensorArray(xyz=t(w.sensors), sound_speed=w.v, fs=w.fs, n_samples=w.Nt, t0=w.t0, window_k=w.k)
    y = torch.empty((w.Nd, w.Nt), device=dev)
    d = torch.randn((w.Nd, w.Nt), device=dev, generator=torch.Generator(device=dev).manual_seed(3))
    gA, gc, gsg = torch.empty(w.M, device=dev), torch.empty((3, w.M), device=dev), torch.empty(w.M, device=dev)
    fns = {"forward": lambda: _lib.gpair_forward(gs, arr, y),
           "adjoint_full": lambda: _lib.gpair_adjoint(gs, arr, d, gA, gc, gsg)}
    times = {}
    reps = max(3, min(args.steps, 10))
    for name, fn in fns.items():
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        times[name] = max_over_ranks(a0.elapsed_time(a1) / reps, world) / 1e3
    assert _lib.gpair_last_device_status() == 0
    pairs = float(w.M) * w.Nd
    mean_sigma = float(np.mean(sg.astype(np.float64)))
    samples = pairs * 2.0 * w.k * mean_sigma * w.fs / w.v
    work = {"forward": (FP32_PER_SAMPLE["forward"] * samples + FP32_PER_PAIR * pairs,
                        MUFU_PER_SAMPLE * samples + MUFU_PER_PAIR * pairs),
            "adjoint_full": (FULL_FP32_PER_SAMPLE * samples + FULL_FP32_PER_PAIR * pairs,
                             FULL_MUFU_PER_SAMPLE * samples + FULL_MUFU_PER_PAIR * pairs)}
    out = {"workload": w.name, "gaussians": w.M, "sensors": w.Nd, "samples": w.Nt, "pairs": pairs,
           "sample_evals": samples, "amplitudes": "dense U[0,1]^2", "reps": reps,
           "kernels": {"forward": "fwd_free_lanes_kernel", "adjoint_full": "adj_kernel (A, c, sigma)"}}
    for name, (F, X) in work.items():
        tm = times[name]
        t_fp32, t_mufu = F / p_fp32, X / p_mufu
        pipe = "fp32" if t_fp32 >= t_mufu else "mufu"
        ops, peak = (F, p_fp32) if pipe == "fp32" else (X, p_mufu)
        pm = pipe_peaks[pipe] * 1e12
        out[name] = {"ms": tm * 1e3, "alg_fp32_ops": F, "alg_mufu_ops": X, "bound_pipe": pipe,
                     "achieved": ops / tm / 1e12, "peak": peak / 1e12, "frac": ops / tm / peak,
                     "frac_of_measured": ops / tm / pm, "pair_evals_per_s": pairs / tm,
                     "includes": ("tile and slab summaries + fwd_free_lanes_kernel + slab reduction" if name == "forward"
                                  else "tile summaries + adj_kernel with centre and width gradients")}
    return out


def warmstart_leg(args):
    """The learned warm start at the mid geometry (128 x 128 x 64 Gaussians, 1024 sensors x 4096
    samples): the BF16 U-Net trained on `ws_train` seeded vessel-tree phantoms whose signals come
    from gpair_forward (the library's kernels do the data, the training and the reconstructions),
    then on `ws_eval` held-out seeds the plain reconstruction (Algorithm 2 from zero, the
    configuration's 50 iterations, its best step size) against A^T b -> network -> the same solver
    until the plain final residual is reached within a relative 1e-3.  Device seconds per
    reconstruction; the one-time training is reported separately (not in warm_s) with the number of
    reconstructions that pays it back."""
    from paper_2602_03893_gb300 import warmstart
    procs = max(1, min(16, len(os.sched_getaffinity(0))))
    t0 = time.perf_counter()
    rep, _ = warmstart.run(n_train=args.ws_train, n_eval=args.ws_eval, n_timed=args.ws_eval, epochs=args.ws_epochs,
                           lr=1e-3, iters=50, procs=procs, log=None)
    wall = time.perf_counter() - t0
    rows = rep["rows"]
    gain = rep["plain_s_mean"] - rep["warm_s_mean"]
    return {"workload": rep["workload"], "n_train": rep["n_train"], "epochs": rep["epochs"], "n_seeds": len(rows),
            "reached_frac": rep["reached_frac"], "plain_s": rep["plain_s_mean"], "warm_s": rep["warm_s_mean"],
            "plain_iters": rep["ir_iters"], "warm_iters_mean": rep["warm_iters_mean"],
            "warm_iters_max": max(r["warm_iters"] for r in rows), "eta_plain": rep["eta"], "eta_warm": rep["eta_warm"],
            "warm_net_s_mean": float(np.mean([r["warm_net_s"] for r in rows])),
            "x0_rel_err_mean": rep["x0_rel_err_mean"], "train_s": rep["train_s"], "data_s": rep["data_s"],
            "train_loss_first": rep["train_loss_first"], "train_loss_last": rep["train_loss_last"],
            "training_included_in_warm_s": False,
            "break_even_reconstructions": (rep["train_s"] / gain) if gain > 0 else None,
            "target": "warm residual <= (1 + 1e-3) x plain residual after 50 iterations", "leg_wall_s": wall}


def src_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2602_03893_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, src, workload):
    """dram bytes per launch from the committed ncu summary, if it was taken on this source and
    this workload."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("src_hash") == src and e.get("workload") == workload:
            return e.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


L2_MB = 129.0    # GB300 L2


def l2_note(w):
    """How the step's operands compare with L2 (no flush is done between timed steps)."""
    vol_mb, rec_mb = 4.0 * w.M / 1e6, 4.0 * w.Nd * w.Nt / 1e6
    step_mb = 5 * vol_mb + 3 * rec_mb     # A-sized z, m, v, x, gradient; y, b and the residual
    kind = "larger than L2" if step_mb > L2_MB else "SMALLER than L2 (cached between steps)"
    return (f"operands {kind} ({L2_MB:.0f} MB): {vol_mb:.1f} MB per volume (z, m, v, x, gradient), "
            f"{rec_mb:.1f} MB per record (y, b, residual), {step_mb:.0f} MB per step without the slab partial rows")


class ClockSampler:
    """nvidia-smi sampling of the device's SM clock and throttle reasons every 200 ms."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def _mine(self):
        mine = [r for r in self.rows if self.uuid and self.uuid.lower() in r[0].lower()]
        return mine or self.rows

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=5)

    def summary(self):
        self.rows = self._mine()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1])]
        mx = [num(r[2]) for r in self.rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in self.rows)}


def cpu_baseline(w, n_sensors, seed=5):
    """The FP64 oracle (as it stands) on a bounded sample: one forward + adjoint over all
    Gaussians and `n_sensors` sensors, extrapolated linearly to all sensors (both operators are
    sums of independent per-sensor terms)."""
    import oracle
    oracle.build()
    threads = len(os.sched_getaffinity(0))
    oracle.set_threads(threads)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.Nd, n_sensors, replace=False))
    sens = np.ascontiguousarray(w.sensors[idx])
    x = (rng.uniform(0.0, 1.0, w.M) ** 2).astype(np.float32)
    G = oracle.gaussians_from_grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.ox, w.grid.oy, w.grid.oz, w.grid.h,
                                   w.grid.sigma, x)
    delta = rng.normal(size=(n_sensors, w.Nt))
    t0 = time.perf_counter()
    oracle.forward(G, sens, w.v, w.fs, w.t0, w.Nt, k=w.k)
    t1 = time.perf_counter()
    oracle.adjoint(G, sens, w.v, w.fs, w.t0, w.Nt, delta, k=w.k)
    t2 = time.perf_counter()
    per_iter = (t2 - t0) * (w.Nd / n_sensors)
    return {"value": per_iter, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one forward + adjoint of all {w.M} Gaussians x {n_sensors} of {w.Nd} sensors "
                      f"({t1 - t0:.1f} s + {t2 - t1:.1f} s), scaled by {w.Nd}/{n_sensors}"}


def dist_setup(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """--impl reference: the oracle (CPU, FP64) timed on this machine's host cores for the same
    metric, each step a bounded sample (a sensor subset) of the workload, scaled to all sensors."""
    if rank != 0:
        return
    w = workload(args.workload)
    # about 370 sensor-operators in total (a few minutes on 16 cores at the paper scale), spread over the
    # warm-up and timed steps, at most cpu_sensors / 2 per step
    ns = max(1, min(w.Nd, args.cpu_sensors // 2, 368 // max(1, args.warmup + args.steps)))
    vals = []
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(w, ns, seed=100 + s)
        if s >= args.warmup:
            vals.append(r["value"])
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "gaussians": w.M, "sensors": w.Nd, "samples": w.Nt,
                       "parallelism": f"replicas{world}"},
            "cpu_baseline": {"kind": "oracle", "cores": r["cores"], "value": v, "unit": UNIT,
                             "sample": f"per step: forward + adjoint over all Gaussians x {ns} sensors, scaled by "
                                       f"{w.Nd}/{ns}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            # the value is extrapolated: each step times ns sensors and scales linearly to all of them
            "extrapolated_from_sensors": ns, "extrapolation_factor": w.Nd / ns,
            "measured_s_per_step": v * ns / w.Nd}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    from paper_2602_03893_gb300 import _lib, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    g = w.grid
    grid = _lib.Grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma)
    A_true = torch.as_tensor(w.A, device=dev)
    arr = _lib.SensorArray(xyz=torch.as_tensor(w.sensors, device=dev), sound_speed=w.v, fs=w.fs, n_samples=w.Nt,
                           t0=w.t0, window_k=w.k)
    # measured data: forward of the phantom + 30 dB noise, scaled to max |b| = 1
    y = torch.empty((w.Nd, w.Nt), device=dev)
    _lib.gpair_forward(_lib.Gaussians(A=A_true, grid=grid), arr, y)
    b_np = synth.add_noise(y.cpu().numpy(), 30.0, seed=7)
    b_np /= np.abs(b_np).max()
    b = torch.as_tensor(b_np, device=dev)
    b_host = torch.as_tensor(b_np).pin_memory()
    b_dev2 = torch.empty_like(b)

    iters_total = args.warmup + args.steps
    params = _lib.StepParams(rule=_lib.RULE_ADAM, npc=1, npc_eps=1e-8, eta_max=0.02, eta_min=0.0,
                             T0=max(1, 2 * iters_total), adam_eps=1e-20)
    gs = _lib.Gaussians(A=A_true, grid=grid)     # the solver's amplitudes are its own iterate
    solver = _lib.Solver(gs, arr, params)
    stream = torch.cuda.current_stream(dev)

    # ---- device-resident timing
    for _ in range(args.warmup):
        solver.gpair_step(b, want_loss=False)
    torch.cuda.synchronize()
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler(str(uuid) if uuid is not None else None)
    sampler.start()
    time.sleep(0.3)
    solver.gpair_solver_profile(True)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.gpair_step(b, want_loss=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    sampler.stop()
    t_ms = e0.elapsed_time(e1)
    (fwd_ms, adj_ms, step_ms), nrec = solver.gpair_solver_timings()
    solver.gpair_solver_profile(False)
    assert _lib.gpair_last_device_status() == 0, "device status word set during the timed region"
    t_max = max_over_ranks(t_ms, world)
    per_iter = t_max / 1e3 / (args.steps * world)

    # ---- end to end through the public API with host buffers
    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        b_dev2.copy_(b_host, non_blocking=True)
        solver.gpair_step(b_dev2, want_loss=True)
    barrier(world)
    torch.cuda.synchronize()
    tw0 = time.perf_counter()
    for _ in range(e2e_steps):
        b_dev2.copy_(b_host, non_blocking=True)          # H2D of the step's input (pinned)
        loss, resid = solver.gpair_step(b_dev2, want_loss=True)   # D2H of the FP64 loss (syncs)
    torch.cuda.synchronize()
    tw = time.perf_counter() - tw0
    tw = max_over_ranks(tw, world)
    e2e = {"value": tw / (e2e_steps * world), "unit": UNIT, "h2d_bytes_per_step": int(b.numel() * 4),
           "d2h_bytes_per_step": 8, "loss_last": loss}

    # ---- the same K steps replayed as one CUDA graph (gpair_solver_steps), device time; the first
    # call captures the graph
    solver.gpair_solver_steps(b, 1, want_loss=False)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    solver.gpair_solver_steps(b, args.steps, want_loss=False)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = max_over_ranks(g0.elapsed_time(g1) / args.steps, world)

    # ---- the paper's own operator (ASSA, Algorithm 1) on the same workload and the solver's image,
    # timed after the IR step; the paper's figures (RTX 5090) are context
    assa = None
    if not args.no_assa:
        x_img = solver.gpair_solver_image()
        gx = _lib.Gaussians(A=x_img, grid=grid)
        ya, ga = torch.empty_like(b), torch.empty_like(x_img)
        ra = torch.randn(b.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
        times = {}
        for name, fn in (("forward", lambda: _lib.gpair_assa_forward(gx, arr, ya, n_min=ASSA_NMIN)),
                         ("adjoint", lambda: _lib.gpair_assa_adjoint(gx, arr, ra, ga, n_min=ASSA_NMIN))):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(args.steps):
                fn()
            a1.record(stream)
            torch.cuda.synchronize()
            times[name] = max_over_ranks(a0.elapsed_time(a1) / args.steps, world)
        # one whole IR iteration (Algorithm 2, same rule and data) with ASSA as the solver's operator
        sa = _lib.Solver(gs, arr, dataclasses.replace(params, op=_lib.OP_ASSA, n_min=ASSA_NMIN))
        for _ in range(2):
            sa.gpair_step(b, want_loss=False)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            sa.gpair_step(b, want_loss=False)
        a1.record(stream)
        torch.cuda.synchronize()
        times["ir_step"] = max_over_ranks(a0.elapsed_time(a1) / args.steps, world)
        sa.close()
        assert _lib.gpair_last_device_status() == 0
        nh = math.ceil(3.0 * float(np.float32(g.sigma)) / (float(np.float32(w.v)) / float(np.float32(w.fs))))
        alpha = max(1, math.ceil(((ASSA_NMIN - 1) / 2.0) / nh))
        assa = {"n_min": ASSA_NMIN, "alpha": alpha, "n_half": nh, "forward_ms": times["forward"],
                "adjoint_ms": times["adjoint"], "fwd_plus_adj_ms": times["forward"] + times["adjoint"],
                "ir_step_ms": times["ir_step"],
                "pair_evals_per_s": 2 * pairs_of(w) / ((times["forward"] + times["adjoint"]) / 1e3),
                "paper_ms": {"forward": 37.41, "adjoint": 4.99, "hardware": "RTX 5090 (the paper's)"},
                "includes": "forward: slab info + kernel + slab reduction; adjoint: correlated residual + kernel; "
                            "ir_step: gpair_step with op = ASSA (NPC, forward, FP64 loss, adjoint, Adam)"}

    # ---- the vessel continuity regulariser (value + gradient) on the same image, HBM-bound
    vcr = None
    if not args.no_assa:
        x_img = solver.gpair_solver_image()
        gv = torch.zeros_like(x_img)
        dims = (g.nz, g.ny, g.nx)
        for _ in range(2):
            _lib.gpair_vcr(x_img, dims, 0.5, 1e-8, 1e-3, gv, want_value=False)
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(args.steps):
            _lib.gpair_vcr(x_img, dims, 0.5, 1e-8, 1e-3, gv, want_value=False)
        v1.record(stream)
        torch.cuda.synchronize()
        vms = v0.elapsed_time(v1) / args.steps
        # one fused pass: x read, gradient read and written, 12 bytes per voxel (the fields stay on chip)
        vbytes = 4.0 * (1 + 2) * w.M
        vcr = {"ms": vms, "alg_bytes": vbytes, "achieved_GBs": vbytes / (vms / 1e3) / 1e9,
               "peak_GBs": HBM_GBS, "frac": vbytes / (vms / 1e3) / 1e9 / HBM_GBS,
               "includes": "vcr_march_kernel (fields in shared memory + transposed-stencil gradient + FP64 "
                           "block partials); no host sync"}

    # ---- voxelization of the image (Eq. 2 sampled on the lattice: three separable gather passes) and
    # the image metrics (MSE, PSNR, SSIM of the iterate against the phantom): HBM-bound passes
    vox = met = None
    if not args.no_assa:
        x_img = solver.gpair_solver_image()
        gxi = _lib.Gaussians(A=x_img, grid=grid)
        vol = torch.empty(w.M, device=dev)
        for _ in range(2):
            _lib.gpair_voxelize(gxi, grid, 3.0, vol)
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(args.steps):
            _lib.gpair_voxelize(gxi, grid, 3.0, vol)
        v1.record(stream)
        torch.cuda.synchronize()
        xms = v0.elapsed_time(v1) / args.steps
        xbytes = 8.0 * w.M      # amplitudes in, volume out
        vox = {"ms": xms, "alg_bytes": xbytes, "achieved_GBs": xbytes / (xms / 1e3) / 1e9, "peak_GBs": HBM_GBS,
               "frac": xbytes / (xms / 1e3) / 1e9 / HBM_GBS,
               "includes": "gpair_voxelize, lattice case: the three separable passes fused in one kernel (the volume read and written once)"}
        dims = (g.nz, g.ny, g.nx)
        rng_max = float(A_true.max())
        vals, times = None, []
        for it in range(2 + args.steps):
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            vals = _lib.gpair_image_metrics(x_img, A_true, dims, 7, rng_max)   # synchronises
            m1.record(stream)
            torch.cuda.synchronize()
            if it >= 2:
                times.append(m0.elapsed_time(m1))
        mms = statistics.median(times)
        mbytes = 8.0 * w.M      # both volumes read once
        met = {"ms": mms, "alg_bytes": mbytes, "achieved_GBs": mbytes / (mms / 1e3) / 1e9, "peak_GBs": HBM_GBS,
               "frac": mbytes / (mms / 1e3) / 1e9 / HBM_GBS, "values": vals, "window": 7,
               "includes": "gpair_image_metrics on the volume: FP64 MSE, separable box sums, SSIM map, "
                           "FP64 mean, result copied to the host"}

    # the two pipes' rates measured on this device right after the timed work (FFMA and ex2 chains)
    pipe_peaks = {"fp32": _lib.gpair_pipe_peak(_lib.PIPE_FP32) / 1e12, "mufu": _lib.gpair_pipe_peak(_lib.PIPE_MUFU) / 1e12,
                  "unit": "T lane-ops/s", "method": "gpair_pipe_peak: 8 dependent-chain FFMA / ex2.approx streams per "
                                                     "thread, 8 CTAs x 256 threads per SM, CUDA events"}

    clocks = sampler.summary()
    pairs, samples = work_units(w)
    fwd_avg = fwd_ms / max(nrec, 1) / 1e3
    adj_avg = adj_ms / max(nrec, 1) / 1e3
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count   # queried, not assumed
    p_fp32 = sm_count * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6
    p_mufu = sm_count * MUFU_LANES_PER_SM * SM_MAX_MHZ * 1e6
    names = kernel_names(w)
    kern = {}
    for op, t in (("forward", fwd_avg), ("adjoint", adj_avg)):
        F, X = alg_work(w, op)
        t_fp32, t_mufu = F / p_fp32, X / p_mufu
        pipe = "fp32" if t_fp32 >= t_mufu else "mufu"
        ops, peak = (F, p_fp32) if pipe == "fp32" else (X, p_mufu)
        pm = pipe_peaks[pipe] * 1e12
        kern[op] = {"kernel": names[op], "s_per_launch": t, "bound_pipe": pipe, "t_bound_s": max(t_fp32, t_mufu),
                    "alg_fp32_ops": F, "alg_mufu_ops": X, "achieved": ops / t / 1e12, "peak": peak / 1e12,
                    "frac": ops / t / peak, "peak_measured": pm / 1e12, "frac_of_measured": ops / t / pm,
                    "t_bound_measured_s": max(F / (pipe_peaks["fp32"] * 1e12), X / (pipe_peaks["mufu"] * 1e12))}
    dom = "forward" if fwd_avg >= adj_avg else "adjoint"
    src = src_hash("forward_lanes.cu" if dom == "forward" else "adjoint.cu", "gpair_internal.cuh")
    tr = profiled_traffic(kern[dom]["kernel"], src, w.name)
    kd = kern[dom]
    roofline = {"bound": "alu", "achieved": kd["achieved"], "peak": kd["peak"],
                "unit": "T lane-ops/s (" + ("FP32" if kd["bound_pipe"] == "fp32" else "MUFU") + ")",
                "frac": kd["frac"], "traffic": tr, "kernel": kd["kernel"],
                "sm_count": sm_count,
                "peak_basis": f"{sm_count} SMs (queried) x {FP32_LANES_PER_SM} FP32 / {MUFU_LANES_PER_SM} MUFU lanes x "
                              f"{SM_MAX_MHZ:.0f} MHz (max SM clock); not in the measured-peaks file",
                "kernels": kern}
    # both operators of the iteration together: their bounds over their measured times
    roofline["fwd_plus_adj_frac"] = ((kern["forward"]["t_bound_s"] + kern["adjoint"]["t_bound_s"]) /
                                     (fwd_avg + adj_avg))
    roofline["fwd_plus_adj_frac_of_measured"] = ((kern["forward"]["t_bound_measured_s"] +
                                                  kern["adjoint"]["t_bound_measured_s"]) / (fwd_avg + adj_avg))
    roofline["pipe_peaks_measured"] = pipe_peaks
    # the dominant kernel's algorithmic bytes per launch, beside the measured traffic: the forward
    # reads the amplitudes and writes y (through its slab partial rows); the adjoint reads the
    # residual and writes the amplitude gradient
    alg_bytes = 4.0 * (w.M + w.Nd * w.Nt)
    roofline["traffic_alg_bytes"] = alg_bytes
    if tr:
        roofline["traffic_over_alg"] = tr / alg_bytes
        roofline["traffic_note"] = ("forward: the amplitudes read once, the rest the slab partial rows (each row "
                                    "its own band of samples), summed into y by the slab reduction"
                                    if dom == "forward" else "adjoint: the residual table is served from L2")
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = kd["frac"] * SM_MAX_MHZ / clocks["sm_mhz"]

    diff = None
    if not args.no_assa:
        diff = diff_leg(args, dev, stream, p_fp32, p_mufu, pipe_peaks, world)
    ws = None
    if not args.no_warmstart and rank == 0 and world == 1:
        ws = warmstart_leg(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, min(args.cpu_sensors, w.Nd))

    if rank == 0:
        line = {"metric": METRIC, "value": per_iter, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "gaussians": w.M, "sensors": w.Nd, "samples": w.Nt,
                           "grid": [g.nx, g.ny, g.nz], "spacing_m": g.h, "sigma_m": g.sigma, "window_k": w.k,
                           "fs_hz": w.fs, "sound_speed": w.v, "step": "Adam + NPC + CAWR, FP64 loss",
                           "l2": l2_note(w),
                           "parallelism": f"replicas{world}"},
                "pair_evals_per_s": 2 * pairs / per_iter, "sample_evals_per_s": 2 * samples / per_iter,
                "kernel_ms": {"forward": fwd_avg * 1e3, "adjoint": adj_avg * 1e3,
                              "step_device": step_ms / max(nrec, 1)},
                "graph_ms_per_step": graph_ms,
                "roofline": roofline, "assa": assa, "vcr": vcr, "voxelize": vox, "metrics": met, "diff": diff, "warmstart": ws,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": LAUNCHES_PER_STEP * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
