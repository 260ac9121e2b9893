"""The operators at the edges of the boundary's documented limits, against the oracle:

- 65535 sensors, the largest count a launch-grid dimension takes;
- a record of 2^23 samples whose windows lie about four million samples in (sensors 150 m
  away).  This checks the FP64 per-(tile, sensor) reference that keeps the FP32 phase offsets
  small, and the fine-sample indexing of the discretised operator (alpha n0 ~ 8e6)."""
import os

import numpy as np
import pytest

import oracle
from gpair_testutil import TAU, assert_signal_parity, gpu_adjoint, gpu_forward, oracle_gaussians
from paper_2602_03893_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)


def _grad_parity(g_gpu, g_ora, amb, tol=1e-4):
    err = np.linalg.norm(np.asarray(g_gpu, np.float64) - g_ora)
    assert np.all(np.isfinite(g_gpu))
    assert err <= tol * np.linalg.norm(g_ora) + np.linalg.norm(amb), err / np.linalg.norm(g_ora)


def test_65535_sensors_forward_and_adjoint():
    g = synth.centred_grid(6, 5, 4, 0.1e-3)
    rng = np.random.default_rng(31)
    A = rng.uniform(0.1, 1.0, g.M).astype(np.float32)
    w = synth.Workload("nd-max", g, synth.cap_sensors(65535, 12e-3, 160.0), 512, A=A)
    G = oracle_gaussians(w)
    y = gpu_forward(w)
    idx = np.concatenate([[0, 1, 32767, 65533, 65534], rng.choice(65535, 59, replace=False)])
    y_ora, amb = oracle.forward(G, w.sensors[idx], w.v, w.fs, w.t0, w.Nt, k=w.k, tau=TAU, want_amb=True)
    assert_signal_parity(y[idx], y_ora, amb)
    delta = rng.normal(size=(w.Nd, w.Nt)).astype(np.float32)
    out = gpu_adjoint(w, delta, full=False)
    ref = oracle.adjoint(G, w.sensors, w.v, w.fs, w.t0, w.Nt, delta, k=w.k, want=("A",), tau=TAU, want_amb=True)
    _grad_parity(out["A"], ref["A"], ref["ambA"])


def _far_workload():
    g = synth.centred_grid(8, 6, 4, 0.1e-3)
    A = np.random.default_rng(32).uniform(0.1, 1.0, g.M).astype(np.float32)
    # only distant sensors: a near one would dominate every norm below
    sens = np.array([[0.0, 0.0, -150.0], [90.0, -40.0, -110.0]], dtype=np.float32)
    return synth.Workload("far", g, sens, 1 << 23, A=A)


def test_long_record_far_sensors_forward_and_adjoint():
    w = _far_workload()
    G = oracle_gaussians(w)
    y = gpu_forward(w)
    y_ora, amb = oracle.forward(G, w.sensors, w.v, w.fs, w.t0, w.Nt, k=w.k, tau=TAU, want_amb=True)
    assert np.count_nonzero(y_ora[0]) > 0 and np.nonzero(y_ora[0])[0].min() > 3_900_000
    for j in range(w.Nd):
        assert_signal_parity(y[j], y_ora[j], amb[j])
    delta = np.random.default_rng(33).normal(size=(w.Nd, w.Nt)).astype(np.float32)
    out = gpu_adjoint(w, delta, full=False)
    ref = oracle.adjoint(G, w.sensors, w.v, w.fs, w.t0, w.Nt, delta, k=w.k, want=("A",), tau=TAU, want_amb=True)
    _grad_parity(out["A"], ref["A"], ref["ambA"])


def test_long_record_far_sensors_discretised_operator():
    import torch

    from gpair_testutil import device_inputs
    from paper_2602_03893_gb300 import _lib

    w = _far_workload()
    G = oracle_gaussians(w)
    gs, arr = device_inputs(w)
    y = torch.full((w.Nd, w.Nt), float("nan"), device="cuda")
    _lib.gpair_assa_forward(gs, arr, y, n_min=25)
    torch.cuda.synchronize()
    assert _lib.gpair_last_device_status() == 0
    y_ora, amb = oracle.assa_forward(G, G.sigma[0], w.sensors, w.v, w.fs, w.t0, w.Nt, n_min=25, tau=1e-4,
                                     want_amb=True)
    yg = y.cpu().numpy()
    for j in range(w.Nd):
        assert_signal_parity(yg[j], y_ora[j], amb[j])
    delta = np.random.default_rng(34).normal(size=(w.Nd, w.Nt)).astype(np.float32)
    gA = torch.full((w.M,), float("nan"), device="cuda")
    _lib.gpair_assa_adjoint(gs, arr, torch.as_tensor(delta, device="cuda"), gA, n_min=25)
    torch.cuda.synchronize()
    g_ora, gamb = oracle.assa_adjoint(G, G.sigma[0], w.sensors, w.v, w.fs, w.t0, w.Nt, delta, n_min=25, tau=1e-4,
                                      want_amb=True)
    _grad_parity(gA.cpu().numpy(), g_ora, gamb)
