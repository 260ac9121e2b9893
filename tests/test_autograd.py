"""Differentiation through the autograd Function (free centres, widths and amplitudes):
gradients against the FP64 oracle, against central finite differences of the FP64 oracle
forward, and a short Adam fit on the 262,144-Gaussian, 512-sensor, 2048-sample workload."""
import os

import numpy as np
import pytest
import torch

import oracle
from gpair_testutil import TAU, device_inputs, oracle_gaussians
from paper_2602_03893_gb300 import autograd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def work():
    oracle.set_threads(os.cpu_count() or 1)
    return synth.differentiable(4)


def _params(w, dev="cuda"):
    cx, cy, cz, sg, A = w.free
    t = lambda q: torch.tensor(q, device=dev, dtype=torch.float32, requires_grad=True)
    return t(A), t(cx), t(cy), t(cz), t(sg)


@pytest.mark.parametrize("k", [3.0, 6.0])
def test_autograd_matches_oracle_gradient(work, k):
    w = work
    _, arr = device_inputs(w, k=k)
    A, cx, cy, cz, sg = _params(w)
    y = autograd.gaussian_signals(A, cx, cy, cz, sg, arr)
    delta = np.random.default_rng(3).normal(size=(w.Nd, w.Nt)).astype(np.float32)
    y.backward(torch.as_tensor(delta, device="cuda"))
    idx = np.sort(np.random.default_rng(4).choice(w.M, 3000, replace=False))
    G = oracle_gaussians(w)
    Gs = oracle.Gaussians(G.c[idx], G.sigma[idx], G.A[idx])
    ref = oracle.adjoint(Gs, w.sensors, w.v, w.fs, w.t0, w.Nt, delta, k=k, want=("A", "c", "sigma"), tau=TAU,
                         want_amb=True)
    got = {"A": A.grad.cpu().numpy()[idx], "sigma": sg.grad.cpu().numpy()[idx],
           "c": np.stack([cx.grad.cpu().numpy()[idx], cy.grad.cpu().numpy()[idx], cz.grad.cpu().numpy()[idx]])}
    for key, amb in (("A", "ambA"), ("c", "ambC"), ("sigma", "ambS")):
        err = np.linalg.norm(got[key] - ref[key])
        assert err <= 1e-4 * np.linalg.norm(ref[key]) + np.linalg.norm(ref[amb]), key


def test_autograd_against_central_fd_of_oracle_forward(work):
    """64 random parameters; central differences (h = 1e-4 relative; centres use 1e-4 sigma)
    of L = <delta, y> evaluated by the FP64 oracle forward of the perturbed Gaussian alone (the
    forward is linear in the Gaussian set).  k = 6 so that the moving window edge carries no
    weight."""
    w = work
    k = 6.0
    _, arr = device_inputs(w, k=k)
    A, cx, cy, cz, sg = _params(w)
    delta = np.random.default_rng(5).normal(size=(w.Nd, w.Nt))
    y = autograd.gaussian_signals(A, cx, cy, cz, sg, arr)
    y.backward(torch.as_tensor(delta.astype(np.float32), device="cuda"))
    grads = [A.grad.cpu().numpy(), cx.grad.cpu().numpy(), cy.grad.cpu().numpy(), cz.grad.cpu().numpy(),
             sg.grad.cpu().numpy()]
    G = oracle_gaussians(w)
    rng = np.random.default_rng(6)
    nz = np.flatnonzero(G.A > 0.05)
    worst = 0.0
    for _ in range(64):
        i = int(rng.choice(nz))
        which = int(rng.integers(0, 5))

        def L(dA=0.0, dc=(0.0, 0.0, 0.0), ds=0.0):
            c = (G.c[i] + np.asarray(dc))[None, :]
            Gi = oracle.Gaussians(c, np.array([G.sigma[i] + ds]), np.array([G.A[i] + dA]))
            return float(np.sum(oracle.forward(Gi, w.sensors, w.v, w.fs, w.t0, w.Nt, k=k) * delta))
        if which == 0:
            h = 1e-4 * G.A[i]
            fd = (L(dA=h) - L(dA=-h)) / (2 * h)
        elif which == 4:
            h = 1e-4 * G.sigma[i]
            fd = (L(ds=h) - L(ds=-h)) / (2 * h)
        else:
            h = 1e-4 * G.sigma[i]
            e = np.zeros(3)
            e[which - 1] = h
            fd = (L(dc=e) - L(dc=-e)) / (2 * h)
        g = grads[which][i]
        scale = max(abs(fd), 1e-3 * np.abs(grads[which]).max())
        worst = max(worst, abs(g - fd) / scale)
    assert worst < 1e-3, worst


def test_adam_fit_of_free_gaussians(work):
    """100 Adam iterations on (A, c, sigma) from a perturbed start towards data from the truth."""
    w = work
    _, arr = device_inputs(w)
    A, cx, cy, cz, sg = _params(w)
    with torch.no_grad():
        b = autograd.gaussian_signals(A, cx, cy, cz, sg, arr).clone()
        gen = torch.Generator(device="cuda").manual_seed(0)
        A.mul_(1 + 0.3 * torch.randn(A.shape, device="cuda", generator=gen)).clamp_(min=0)
        cx.add_(2e-5 * torch.randn(cx.shape, device="cuda", generator=gen))
        sg.mul_(1.1)
    opt = torch.optim.Adam([{"params": [A], "lr": 1e-2}, {"params": [cx, cy, cz], "lr": 2e-6},
                            {"params": [sg], "lr": 2e-6}])
    losses = []
    for _ in range(100):
        opt.zero_grad()
        loss = torch.mean((autograd.gaussian_signals(A, cx, cy, cz, sg, arr) - b) ** 2)
        loss.backward()
        opt.step()
        with torch.no_grad():
            sg.clamp_(min=1e-5)
        losses.append(float(loss.detach()))
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_grid_function_amplitude_gradient_is_adjoint():
    w = synth.tiny(1)
    gs, arr = device_inputs(w)
    A = torch.tensor(np.random.default_rng(1).uniform(0, 1, w.M), device="cuda", dtype=torch.float32,
                     requires_grad=True)
    y = autograd.grid_signals(A, gs.grid, arr)
    d = torch.randn_like(y)
    (y * d).sum().backward()
    from paper_2602_03893_gb300 import _lib
    gA = torch.empty(w.M, device="cuda")
    _lib.gpair_adjoint(_lib.Gaussians(A=A.detach(), grid=gs.grid), arr, d.contiguous(), gA)
    assert torch.allclose(A.grad, gA)
