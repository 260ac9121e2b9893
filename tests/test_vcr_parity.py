"""Vessel continuity regulariser (Methods: R_VCR = R_H + beta R_TV; Algorithm 2's lambda term):
gpair_vcr against the FP64 oracle (value and gradient), and gpair_step with the regulariser
against Algorithm 2 assembled from the oracle's forward, adjoint, regulariser, Adam and CAWR.

Tolerances: value relative 1e-6 (FP32 per voxel, FP64 sum); gradient relative L2 1e-5 on images
whose differences are far above sqrt(eps) (where they are not, the FP32 differences of O(1)
values, ~1e-7, are amplified by up to 1 / sqrt(eps) in the weights, an error of the FP32
evaluation itself); the regularised IR iterates as the plain IR test (2e-3 after a few steps)."""
import os

import numpy as np
import pytest
import torch

import oracle
from gpair_testutil import device_inputs, oracle_gaussians, rel_l2
from oracle import vcr
from paper_2602_03893_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(5, 6, 7), (1, 4, 9), (2, 2, 2), (16, 12, 10), (3, 1, 5)])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_value_and_gradient(dims, beta):
    rng = np.random.default_rng(hash(dims) % 1000)
    x = rng.uniform(0.1, 1.0, dims).astype(np.float32)
    g0 = rng.normal(size=dims).astype(np.float32)
    lam = 0.7
    val_o, g_o = vcr.value_and_grad(x.astype(np.float64), beta)
    xt = torch.as_tensor(x, device="cuda")
    gt = torch.as_tensor(g0, device="cuda")
    val = _lib.gpair_vcr(xt, dims, beta, 1e-8, lam, gt)
    torch.cuda.synchronize()
    assert abs(val - val_o) <= 1e-6 * val_o
    expect = g0.astype(np.float64) + lam * g_o
    assert rel_l2(gt.cpu().numpy() - g0, expect - g0) < 1e-5


def test_value_only_leaves_no_gradient_and_zero_lambda():
    dims = (4, 5, 6)
    x = np.random.default_rng(1).uniform(0, 1, dims).astype(np.float32)
    xt = torch.as_tensor(x, device="cuda")
    gt = torch.zeros(dims, device="cuda")
    v1 = _lib.gpair_vcr(xt, dims, 0.3)
    v2 = _lib.gpair_vcr(xt, dims, 0.3, lam=0.0, grad=gt)
    assert v1 == v2
    assert torch.count_nonzero(gt).item() == 0


def test_regularised_step_matches_oracle_algorithm_2():
    oracle.set_threads(os.cpu_count() or 1)
    w = synth.tiny(1)
    G = oracle_gaussians(w)
    y = oracle.forward(G, w.sensors, w.v, w.fs, w.t0, w.Nt, k=w.k)
    b = synth.add_noise(y.astype(np.float32), 30.0, seed=101)
    b = (b / np.abs(b).max()).astype(np.float32)
    iters, eta, lam, beta, eps_n = 5, 0.02, 1e-6, 0.5, 1e-8   # lambda R comparable to the data loss
    dims = (w.grid.nz, w.grid.ny, w.grid.nx)
    z0 = np.random.default_rng(3).uniform(0.2, 1.0, w.M).astype(np.float32)   # warm start: a non-flat image
    p = _lib.StepParams(rule=_lib.RULE_ADAM, npc=1, npc_eps=eps_n, eta_max=eta, eta_min=0.0, T0=iters, T_mult=1.0,
                        adam_eps=1e-20, vcr_lambda=lam, vcr_beta=beta, vcr_eps=1e-8)
    gs, arr = device_inputs(w)
    s = _lib.Solver(gs, arr, p)
    s.gpair_solver_set_state(z=torch.as_tensor(z0, device="cuda"), t=0)
    bt = torch.as_tensor(b, device="cuda")
    loss = np.array([s.gpair_step(bt)[0] for _ in range(iters)])
    x = s.gpair_solver_image().cpu().numpy()
    s.close()
    # Algorithm 2 with the oracle's pieces (FP64)
    N = w.Nd * w.Nt
    z = z0.astype(np.float64)
    m, v = np.zeros_like(z), np.zeros_like(z)
    lo = []
    for t in range(iters):
        xo = (z + eps_n) ** 2
        r = oracle.forward(oracle.Gaussians(G.c, G.sigma, xo), w.sensors, w.v, w.fs, w.t0, w.Nt, k=w.k) - b
        R, gR = vcr.value_and_grad(xo.reshape(dims), beta)
        lo.append(np.sum(r * r) / N + lam * R)
        gx = oracle.adjoint(oracle.Gaussians(G.c, G.sigma, xo), w.sensors, w.v, w.fs, w.t0, w.Nt, 2.0 * r / N,
                            k=w.k)["A"] + lam * gR.ravel()
        oracle.adam(z, m, v, gx * 2.0 * (z + eps_n), t + 1, oracle.cawr(t, eta, 0.0, iters), eps=1e-20)
    xo = (z + eps_n) ** 2
    lo = np.array(lo)
    assert abs(loss[0] - lo[0]) <= 1e-5 * lo[0]
    assert np.max(np.abs(loss - lo) / lo) < 2e-3
    assert rel_l2(x, xo) < 2e-3
    assert lo[-1] < lo[0]


def test_regulariser_requires_grid_and_adam():
    g = synth.centred_grid(4, 4, 4, 0.1e-3)
    w = synth.Workload("free", g, synth.cap_sensors(8, 10e-3, 120.0), 256,
                       free=synth.free_gaussians(g, 3, A=np.ones(g.M)))
    gs, arr = device_inputs(w)
    with pytest.raises(_lib.GpairError):
        _lib.Solver(gs, arr, _lib.StepParams(rule=_lib.RULE_ADAM, vcr_lambda=1e-3, vcr_beta=0.5))
    w2 = synth.tiny(1)
    gs2, arr2 = device_inputs(w2)
    with pytest.raises(_lib.GpairError):
        _lib.Solver(gs2, arr2, _lib.StepParams(rule=_lib.RULE_GD_LINESEARCH, npc=0, vcr_lambda=1e-3))


def test_paper_scale_gradient_at_sampled_voxels():
    """The benchmark's 256 x 256 x 128 volume (16384 tiles, visited in permuted order).  The
    gradient at a voxel depends on x within two voxels per axis, so the oracle evaluates it on the
    crop of +-3 voxels around each sample, which is flush with the volume where it meets a face;
    the samples include faces, edges and corners."""
    nz, ny, nx = 128, 256, 256
    rng = np.random.default_rng(21)
    x = rng.uniform(0.1, 1.0, (nz, ny, nx)).astype(np.float32)
    beta, lam = 0.5, 1.0
    xt = torch.as_tensor(x, device="cuda")
    gt = torch.zeros_like(xt)
    _lib.gpair_vcr(xt, (nz, ny, nx), beta, 1e-8, lam, gt)
    g = gt.cpu().numpy()
    pts = [tuple(int(rng.integers(0, n)) for n in (nz, ny, nx)) for _ in range(60)]
    pts += [(0, 5, 7), (nz - 1, 100, 3), (50, 0, 200), (60, ny - 1, 1), (10, 20, 0), (11, 21, nx - 1),
            (0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, 17), (nz - 1, 0, nx - 1), (64, 128, 31), (64, 3, 32)]
    got, ref = [], []
    for p in pts:
        sl = tuple(slice(max(c - 3, 0), min(c + 4, n)) for c, n in zip(p, (nz, ny, nx)))
        _, gc = vcr.value_and_grad(x[sl].astype(np.float64), beta)
        ref.append(lam * gc[tuple(c - s.start for c, s in zip(p, sl))])
        got.append(g[p])
    assert rel_l2(np.array(got), np.array(ref)) < 1e-5
