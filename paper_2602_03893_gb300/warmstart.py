"""Learned warm start for the reconstruction: training on phantom/signal pairs made by the
library's own forward operator, and the comparison of warm start + iterative reconstruction
against the plain reconstruction from zero (Algorithm 2 from z = 0).

    python -m paper_2602_03893_gb300.warmstart --train 2000 --eval 200 --epochs 2 --out report.json

Workload: the mid geometry (128 x 128 x 64 Gaussians on a 0.1 mm grid, 1024 sensors on a
120-degree cap of radius 60 mm, 4096 samples at 40 MHz), seeded vessel-tree phantoms (training
seeds 1000..., held-out seeds 9000...), measured data = forward + 30 dB white noise.
The network input is A^T b (gpair_adjoint); its output, clamped at 0, is the initial amplitude
image x0 and z0 = sqrt(x0) seeds the NPC parameterisation.  The comparison: plain IR runs
`iters` iterations from zero and records its final residual |Ax - b|; the warm start runs the
same solver from z0 until its residual is within a relative 1e-3 of that value; both are timed on
the device (the warm start including A^T b and the network).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import time

import numpy as np
import torch

from . import _lib, synth, unet


def _phantom(args):
    grid, seed = args
    return synth.vessel_tree_phantom(grid, seed, n_roots=6, max_segments=1200)


def phantoms(grid, seeds, procs=8):
    """Vessel-tree amplitudes for each seed (CPU, spawn-started worker processes)."""
    if procs <= 1 or len(seeds) < 4:
        return [_phantom((grid, s)) for s in seeds]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_phantom, [(grid, s) for s in seeds], chunksize=4)


class Problem:
    """Geometry on the device plus the operators used to make data."""

    def __init__(self, w: synth.Workload):
        self.w = w
        g = w.grid
        self.grid = _lib.Grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma)
        self.arr = _lib.SensorArray(xyz=torch.as_tensor(w.sensors, device="cuda"), sound_speed=w.v, fs=w.fs,
                                    n_samples=w.Nt, t0=w.t0, window_k=w.k)
        self.dims = (g.nz, g.ny, g.nx)
        self.M = g.M

    def forward(self, A):
        y = torch.empty((self.w.Nd, self.w.Nt), device="cuda")
        _lib.gpair_forward(_lib.Gaussians(A=A, grid=self.grid), self.arr, y)
        return y

    def adjoint(self, b):
        g = torch.empty(self.M, device="cuda")
        _lib.gpair_adjoint(_lib.Gaussians(A=g, grid=self.grid), self.arr, b, g)
        return g

    def measure(self, A, seed, snr_db=30.0):
        y = self.forward(A)
        gen = torch.Generator(device="cuda").manual_seed(int(seed))
        sd = math.sqrt(float(torch.mean(y.double() ** 2)) / 10 ** (snr_db / 10))
        return y + sd * torch.randn(y.shape, device="cuda", generator=gen)


def make_set(prob: Problem, seeds, procs=8, keep_signals=True):
    A_list = phantoms(prob.w.grid, list(seeds), procs)
    xs, ts, bs = [], [], []
    for s, A in zip(seeds, A_list):
        At = torch.as_tensor(A, device="cuda")
        b = prob.measure(At, seed=s)
        xs.append(prob.adjoint(b))
        ts.append(At)
        if keep_signals:
            bs.append(b)
    return xs, ts, bs


def train(net: unet.UNet3D, xs, ts, epochs, lr, in_scale, seed=0, log=None):
    order = np.random.default_rng(seed)
    n = len(xs)
    hist = []
    steps = epochs * n
    for e in range(epochs):
        perm = order.permutation(n)
        tot = 0.0
        for q, i in enumerate(perm):
            step = e * n + q
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / steps))      # cosine decay
            loss = net.train_step(xs[i], ts[i], lr_t, in_scale)
            if q % 64 == 0 or q == n - 1:
                tot = float(loss.item()) / net.nv[0]
                hist.append(tot)
                if log:
                    log(f"epoch {e} step {q} loss {tot:.5f}")
    return hist


def reconstruct(prob: Problem, b, iters, eta, z0=None, stop_resid=None):
    """Algorithm 2 through the solver.  Returns (x, residual history, device seconds)."""
    params = _lib.StepParams(rule=_lib.RULE_ADAM, npc=1, npc_eps=1e-8, eta_max=eta, eta_min=0.0, T0=iters,
                             T_mult=1.0, adam_eps=1e-20)
    gs = _lib.Gaussians(A=torch.empty(prob.M, device="cuda"), grid=prob.grid)   # amplitudes: the solver's own
    s = _lib.Solver(gs, prob.arr, params)
    if z0 is not None:
        s.gpair_solver_set_state(z=z0, t=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hist = []
    torch.cuda.synchronize()
    e0.record()
    for it in range(iters):
        loss, resid = s.gpair_step(b)
        hist.append(resid)
        if stop_resid is not None and resid <= stop_resid:
            break
    e1.record()
    torch.cuda.synchronize()
    x = s.gpair_solver_image()
    s.close()
    return x, hist, e0.elapsed_time(e1) / 1e3


def evaluate(prob, net, xs, ts, bs, in_scale, iters, eta, eta_warm):
    rows = []
    for x_in, tgt, b in zip(xs, ts, bs):
        # plain IR from zero
        _, hp, tp = reconstruct(prob, b, iters, eta)
        r_plain = hp[-1]
        # warm start: A^T b and the network (timed), then IR until the plain residual is reached
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aty = prob.adjoint(b)
        x0 = net.predict(aty, in_scale, 1.0, relu=True)
        z0 = torch.sqrt(x0)
        e1.record()
        torch.cuda.synchronize()
        t_net = e0.elapsed_time(e1) / 1e3
        xw, hw, tw = reconstruct(prob, b, iters, eta_warm, z0=z0, stop_resid=(1 + 1e-3) * r_plain)
        # the initial image's own quality
        err0 = float(torch.linalg.norm(x0 - tgt) / torch.linalg.norm(tgt))
        rows.append({"plain_iters": len(hp), "plain_s": tp, "plain_resid": r_plain,
                     "warm_iters": len(hw), "warm_s": tw + t_net, "warm_net_s": t_net, "warm_resid": hw[-1],
                     "reached": hw[-1] <= (1 + 1e-3) * r_plain, "x0_rel_err": err0})
    return rows


def best_eta(prob, b, iters, etas):
    """Step size of the plain reconstruction: the one with the lowest final residual on `b`."""
    res = {eta: reconstruct(prob, b, iters, eta)[1][-1] for eta in etas}
    return min(res, key=res.get), res


def best_eta_warm(prob, net, x_in, b, in_scale, iters, target, etas):
    """Step size of the warm-started reconstruction: fewest iterations to `target` on one sample."""
    x0 = net.predict(x_in, in_scale, 1.0, relu=True)
    z0 = torch.sqrt(x0)
    res = {}
    for eta in etas:
        _, h, _ = reconstruct(prob, b, iters, eta, z0=z0, stop_resid=target)
        res[eta] = (len(h) if h[-1] <= target else iters + 1, h[-1])
    return min(res, key=lambda e: res[e]), {str(k): v for k, v in res.items()}


def run(n_train=2000, n_eval=200, n_timed=None, epochs=2, lr=1e-3, iters=50, eta=None, eta_warm=None,
        workload="mid", procs=8, log=print, seed=0, etas=(0.01, 0.02, 0.05, 0.1, 0.2)):
    w = {"mid": synth.mid, "tiny": synth.tiny}[workload]()
    prob = Problem(w)
    t0 = time.time()
    xs, ts, _ = make_set(prob, range(1000, 1000 + n_train), procs, keep_signals=False)
    t_data = time.time() - t0
    in_scale = 1.0 / float(torch.sqrt(torch.mean(torch.stack([torch.mean(x.double() ** 2) for x in xs]))))
    net = unet.UNet3D(prob.dims, seed=seed)
    torch.cuda.synchronize()
    t1 = time.time()
    hist = train(net, xs, ts, epochs, lr, in_scale, seed=seed, log=log)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    del xs, ts
    ex, et, eb = make_set(prob, range(9000, 9000 + n_eval), procs)
    sweep = sweep_w = None
    if eta is None:   # give the plain reconstruction its best step size (tuned on a held-out sample)
        eta, sweep = best_eta(prob, eb[-1], iters, etas)
    if eta_warm is None:   # and the warm start its own, on the same sample and target
        target = (1 + 1e-3) * reconstruct(prob, eb[-1], iters, eta)[1][-1]
        eta_warm, sweep_w = best_eta_warm(prob, net, ex[-1], eb[-1], in_scale, iters, target, etas)
    # image error of the network alone on every held-out seed
    errs = []
    for x_in, tgt in zip(ex, et):
        x0 = net.predict(x_in, in_scale, 1.0, relu=True)
        errs.append(float(torch.linalg.norm(x0 - tgt) / torch.linalg.norm(tgt)))
    k = n_eval if n_timed is None else min(n_timed, n_eval)
    rows = evaluate(prob, net, ex[:k], et[:k], eb[:k], in_scale, iters, eta, eta_warm)
    rep = {"workload": w.name, "n_train": n_train, "n_eval": n_eval, "n_timed": k, "epochs": epochs,
           "data_s": t_data, "train_s": t_train, "train_steps": epochs * n_train,
           "train_loss_first": hist[0], "train_loss_last": hist[-1], "in_scale": in_scale,
           "x0_rel_err_mean": float(np.mean(errs)), "ir_iters": iters, "eta": eta, "eta_warm": eta_warm,
           "eta_sweep_final_resid": sweep, "eta_warm_sweep_iters_resid": sweep_w,
           "plain_s_mean": float(np.mean([r["plain_s"] for r in rows])),
           "warm_s_mean": float(np.mean([r["warm_s"] for r in rows])),
           "warm_iters_mean": float(np.mean([r["warm_iters"] for r in rows])),
           "reached_frac": float(np.mean([r["reached"] for r in rows])), "rows": rows}
    return rep, net


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--timed", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--eta", type=float, default=None, help="plain-IR step; default: best of a sweep")
    ap.add_argument("--eta-warm", type=float, default=None, help="warm-start step; default: best of a sweep")
    ap.add_argument("--procs", type=int, default=8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    rep, _ = run(a.train, a.eval, a.timed, a.epochs, a.lr, a.iters, a.eta, a.eta_warm, procs=a.procs)
    s = json.dumps(rep)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    summary = {k: v for k, v in rep.items() if k != "rows"}
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
