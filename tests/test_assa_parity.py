"""The paper's discretised operator (adaptive supersampling alignment, Algorithm 1): CUDA path
through the C ABI against the FP64 oracle's three-stage evaluation, element by element.

Snapping a time of flight to the fine grid is an integer decision taken from an FP32 phase on the
GPU and an FP64 distance in the oracle; pairs within TAU_SNAP fine samples of a rounding tie may
go either way, and the oracle bounds what either choice changes (`amb`).  Tolerances: signals
relative L2 1e-5, gradients 1e-4, each plus that bound."""
import os

import numpy as np
import pytest

import oracle
from gpair_testutil import device_inputs, oracle_gaussians, rel_l2
from paper_2602_03893_gb300 import synth

pytestmark = pytest.mark.gpu

TAU_SNAP = 1e-4      # fine samples; the FP32 phase resolves ~1e-6 of one


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)


def gpu_assa_forward(w, A=None, n_min=25):
    import torch

    from paper_2602_03893_gb300 import _lib

    gs, arr = device_inputs(w, A)
    y = torch.full((w.Nd, w.Nt), float("nan"), device="cuda")
    _lib.gpair_assa_forward(gs, arr, y, n_min=n_min)
    torch.cuda.synchronize()
    assert _lib.gpair_last_device_status() == 0
    return y.cpu().numpy()


def gpu_assa_adjoint(w, delta, A=None, n_min=25):
    import torch

    from paper_2602_03893_gb300 import _lib

    gs, arr = device_inputs(w, A)
    d = torch.as_tensor(np.ascontiguousarray(delta, dtype=np.float32), device="cuda")
    gA = torch.full((w.M,), float("nan"), device="cuda")
    _lib.gpair_assa_adjoint(gs, arr, d, gA, n_min=n_min)
    torch.cuda.synchronize()
    return gA.cpu().numpy()


def _check_forward(w, A=None, n_min=25, sensors_idx=None, tol=1e-5):
    G = oracle_gaussians(w, A)
    sens = w.sensors if sensors_idx is None else w.sensors[sensors_idx]
    y_ora, amb = oracle.assa_forward(G, G.sigma[0], sens, w.v, w.fs, w.t0, w.Nt, n_min=n_min, tau=TAU_SNAP,
                                     want_amb=True)
    y = gpu_assa_forward(w, A, n_min)
    if sensors_idx is not None:
        y = y[sensors_idx]
    assert np.all(np.isfinite(y))
    err = np.linalg.norm(y - y_ora)
    assert np.abs(y_ora).max() > 0
    assert err <= tol * np.linalg.norm(y_ora) + np.linalg.norm(amb), (err / np.linalg.norm(y_ora), np.linalg.norm(amb))
    return err / np.linalg.norm(y_ora)


def _dense(w, seed=8):
    return np.random.default_rng(seed).uniform(0.0, 1.0, w.M).astype(np.float32)


@pytest.mark.parametrize("n_min", [25, 101])
def test_tiny_forward(n_min):
    w = synth.tiny(1)
    _check_forward(w, n_min=n_min)
    _check_forward(w, A=_dense(w), n_min=n_min)


def test_tiny_adjoint_and_identity():
    w = synth.tiny(1)
    rng = np.random.default_rng(3)
    delta = rng.normal(size=(w.Nd, w.Nt)).astype(np.float32)
    G = oracle_gaussians(w)
    g_ora, amb = oracle.assa_adjoint(G, G.sigma[0], w.sensors, w.v, w.fs, w.t0, w.Nt, delta, tau=TAU_SNAP,
                                     want_amb=True)
    g = gpu_assa_adjoint(w, delta)
    assert np.all(np.isfinite(g))
    assert np.linalg.norm(g - g_ora) <= 1e-4 * np.linalg.norm(g_ora) + np.linalg.norm(amb)
    # <F x, d> = <x, F^T d> on the GPU itself
    x = _dense(w, 9)
    Fx = gpu_assa_forward(w, A=x).astype(np.float64)
    lhs, rhs = float(np.sum(Fx * delta)), float(x.astype(np.float64) @ g.astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Fx) * np.linalg.norm(delta)


def test_ragged_grid_without_tma_and_time_origin():
    g = synth.centred_grid(13, 11, 7, 0.15e-3)
    A = np.random.default_rng(5).uniform(0.1, 1.0, g.M).astype(np.float32)
    w = synth.Workload("ragged", g, synth.cap_sensors(13, 12e-3, 170.0), 437, A=A, t0=6.4e-6)
    _check_forward(w)
    delta = np.random.default_rng(6).normal(size=(w.Nd, w.Nt)).astype(np.float32)
    G = oracle_gaussians(w)
    g_ora, amb = oracle.assa_adjoint(G, G.sigma[0], w.sensors, w.v, w.fs, w.t0, w.Nt, delta, tau=TAU_SNAP,
                                     want_amb=True)
    gg = gpu_assa_adjoint(w, delta)
    assert np.linalg.norm(gg - g_ora) <= 1e-4 * np.linalg.norm(g_ora) + np.linalg.norm(amb)


def test_mid_sensor_subset():
    w = synth.mid(2)
    idx = np.random.default_rng(0).choice(w.Nd, 10, replace=False)
    _check_forward(w, A=_dense(w), sensors_idx=idx)


def test_paper_scale_full_launch_sampled_sensors():
    """The benchmark's configuration with a dense iterate-like image; the oracle recomputes 6
    sensors (the forward is separable per sensor)."""
    w = synth.paper_scale(3)
    x = (np.random.default_rng(1).uniform(0.0, 1.0, w.M) ** 2).astype(np.float32)
    _check_forward(w, A=x, sensors_idx=np.array([0, 137, 511, 600, 901, 1023]))


def test_free_gaussians_are_rejected():
    from paper_2602_03893_gb300 import _lib

    g = synth.centred_grid(4, 4, 4, 0.1e-3)
    w = synth.Workload("free", g, synth.cap_sensors(8, 10e-3, 120.0), 256,
                       free=synth.free_gaussians(g, 3, A=np.ones(g.M)))
    with pytest.raises(_lib.GpairError):
        gpu_assa_forward(w)


def test_sensor_inside_a_slab_box_and_wide_amplitude_range():
    """The band adds are 32-bit fixed point scaled per (slab, sensor) by the sensor's distance to
    the slab's box; a sensor inside the box keeps float adds.  Amplitudes spanning six decades
    check that rounding to 2^-19 of the largest scaled mass stays within the tolerance."""
    g = synth.centred_grid(16, 12, 8, 0.1e-3)
    rng = np.random.default_rng(12)
    A = (10.0 ** rng.uniform(-6.0, 0.0, g.M)).astype(np.float32)
    sens = synth.cap_sensors(12, 8e-3, 150.0)
    inside = np.array([[0.23e-3, -0.17e-3, 0.11e-3]], dtype=np.float32)     # within the grid's box
    w = synth.Workload("inside", g, np.concatenate([sens, inside]), 512, A=A)
    _check_forward(w, A=A)


def test_paper_scale_adjoint_sampled_gaussians():
    """The benchmark's launch (8.4 M Gaussians x 1024 sensors, alpha = 2); the oracle recomputes
    2000 sampled Gaussians' gradients over all sensors (each entry is independent)."""
    w = synth.paper_scale(3)
    rng = np.random.default_rng(13)
    delta = rng.normal(size=(w.Nd, w.Nt)).astype(np.float32)
    idx = np.sort(rng.choice(w.M, 2000, replace=False))
    g = gpu_assa_adjoint(w, delta)
    assert np.all(np.isfinite(g))
    G = oracle_gaussians(w)
    Gs = oracle.Gaussians(G.c[idx], G.sigma[idx], G.A[idx])
    g_ora, amb = oracle.assa_adjoint(Gs, G.sigma[0], w.sensors, w.v, w.fs, w.t0, w.Nt, delta, tau=TAU_SNAP,
                                     want_amb=True)
    assert np.linalg.norm(g[idx] - g_ora) <= 1e-4 * np.linalg.norm(g_ora) + np.linalg.norm(amb)
