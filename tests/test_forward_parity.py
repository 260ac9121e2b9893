"""Forward operator: CUDA path (through the C ABI) against the FP64 oracle, element by element
on the same seeded inputs.  Tolerance: relative L2 1e-5, plus the weight of terms whose window
decision is ambiguous at FP32 resolution (|d| within TAU of k sigma)."""
import os

import numpy as np
import pytest

import oracle
from gpair_testutil import TAU, assert_signal_parity, edge_workload, gpu_forward, oracle_gaussians, rel_l2
from paper_2602_03893_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)


def _check(w, k=None, A=None, sensors_idx=None):
    k = w.k if k is None else k
    G = oracle_gaussians(w, A)
    y = gpu_forward(w, A=A, k=k)
    sens = w.sensors if sensors_idx is None else w.sensors[sensors_idx]
    y_ora, amb = oracle.forward(G, sens, w.v, w.fs, w.t0, w.Nt, k=k, tau=TAU, want_amb=True)
    yg = y if sensors_idx is None else y[sensors_idx]
    return assert_signal_parity(yg, y_ora, amb), yg, y_ora


@pytest.mark.parametrize("k", [3.0, 6.0])
def test_tiny_phantom(k):
    rel, y, yo = _check(synth.tiny(1), k=k)
    assert np.abs(yo).max() > 0


def test_tiny_dense_amplitudes():
    w = synth.tiny(1)
    A = np.random.default_rng(8).uniform(0.0, 1.0, w.M).astype(np.float32)
    _check(w, A=A)


@pytest.mark.parametrize("sigma_scale", [1.01, 1.02])
def test_window_edge_position_in_and_out_of_expansion(sigma_scale):
    """The sub-sample expansion covers the edge position E when it is inside the window for most
    pairs and corrects the others directly, else leaves E to the direct term; one case each."""
    w = edge_workload(sigma_scale)
    X = 2 * w.k * w.grid.sigma * w.fs / w.v
    assert (X % 1.0 > 0.5) == (sigma_scale > 1.015)
    _check(w)


@pytest.mark.parametrize("h", [0.2e-3, 0.08e-3])
def test_moment_expansion_with_seven_and_eight_terms(h):
    """Delta / sigma = 0.19 keeps 7 terms of the sub-sample expansion; 0.47 needs all 8."""
    g = synth.centred_grid(16, 16, 12, h)
    A = np.random.default_rng(13).uniform(0.0, 1.0, g.M).astype(np.float32)
    w = synth.Workload("terms", g, synth.cap_sensors(64, 20e-3, 160.0), 1024, A=A)
    _check(w)


def test_free_gaussians_per_gaussian_sigma():
    g = synth.centred_grid(24, 20, 16, 0.1e-3)
    free = synth.free_gaussians(g, 31, A=np.random.default_rng(3).uniform(0, 1, g.M))
    w = synth.Workload("free-small", g, synth.cap_sensors(40, 30e-3, 150.0), 2048, free=free)
    for k in (3.0, 6.0):
        _check(w, k=k)


@pytest.mark.parametrize("t0,nt,cut", [(6.4e-6, 437, False), (7.9e-6, 37, True)])
def test_ragged_shapes_and_time_origin(t0, nt, cut):
    """nx not a multiple of 4 (no TMA descriptor), sensors not a multiple of 8, N_t not a
    multiple of 4 and a non-zero t0; in the second case the record is shorter than the arrivals,
    so every sensor's signal is cut at both ends of the record."""
    g = synth.centred_grid(13, 11, 7, 0.15e-3)
    A = np.random.default_rng(5).uniform(0.1, 1.0, g.M).astype(np.float32)
    sens = synth.cap_sensors(13, 12e-3, 170.0)
    w = synth.Workload("ragged", g, sens, nt, A=A, t0=t0)
    rel, y, yo = _check(w)
    # the same sensors over a record extended by `pad` samples on both sides (oracle only)
    pad = 200
    ye = oracle.forward(oracle_gaussians(w), w.sensors, w.v, w.fs, t0 - pad / w.fs, nt + 2 * pad, k=w.k)
    np.testing.assert_allclose(ye[:, pad:pad + nt], yo, rtol=0, atol=1e-12 * np.abs(yo).max())
    outside = np.linalg.norm(ye[:, :pad]) + np.linalg.norm(ye[:, pad + nt:])
    if cut:
        assert np.linalg.norm(ye[:, :pad]) > 0.1 * np.linalg.norm(yo)
        assert np.linalg.norm(ye[:, pad + nt:]) > 0.01 * np.linalg.norm(yo)
        assert np.count_nonzero(y[:, 0]) >= 12 and np.count_nonzero(y[:, -1]) >= 10
    else:
        assert outside == 0.0


def test_edge_cases_single_gaussian_and_empty_window():
    g = synth.centred_grid(1, 1, 1, 0.1e-3)
    w = synth.Workload("one", g, synth.cap_sensors(1, 5e-3, 10.0), 256, A=np.ones(1, np.float32))
    _check(w)
    # every arrival after the last sample: the output is exactly zero
    w2 = synth.Workload("late", g, synth.cap_sensors(3, 50e-3, 10.0), 64, A=np.ones(1, np.float32))
    y = gpu_forward(w2)
    assert np.all(y == 0.0)
    # all-zero amplitudes
    w3 = synth.tiny(1)
    y3 = gpu_forward(w3, A=np.zeros(w3.M, np.float32))
    assert np.all(y3 == 0.0)


def test_mid_sensor_subset():
    w = synth.mid(2)
    idx = np.random.default_rng(0).choice(w.Nd, 12, replace=False)
    rel, _, _ = _check(w, sensors_idx=idx)
    assert rel < 1e-5


def test_paper_scale_full_launch_sampled_sensors_dense_x():
    """The benchmark's configuration (8.4 M Gaussians, 1024 sensors, 4096 samples) with a dense
    iterate-like x; the oracle recomputes 6 sampled sensors exactly (the forward is separable
    per sensor)."""
    w = synth.paper_scale(3)
    x = (np.random.default_rng(1).uniform(0.0, 1.0, w.M) ** 2).astype(np.float32)
    idx = np.array([0, 137, 511, 600, 901, 1023])
    rel, _, _ = _check(w, A=x, sensors_idx=idx)
    assert rel < 1e-5


def test_deterministic_given_inputs_up_to_atomic_order():
    w = synth.tiny(1)
    y1 = gpu_forward(w)
    y2 = gpu_forward(w)
    assert rel_l2(y1, y2) < 1e-6


def test_free_gaussians_band_longer_than_shared_memory():
    """Free Gaussians scattered through an 80 mm cube and sensors 200 mm away: a sensor's samples
    for one slab (2000 to 3700) outnumber the shared signal band (1684 with one warp), so the
    sensor-lane kernel takes two or three passes over each slab, each keeping its own samples (windows
    that lie wholly in another pass's samples add nothing to this one)."""
    rng = np.random.default_rng(21)
    n = 1024
    c = rng.uniform(-40e-3, 40e-3, (3, n))
    free = tuple(np.ascontiguousarray(q, dtype=np.float32) for q in
                 (c[0], c[1], c[2], np.exp(rng.uniform(np.log(0.05e-3), np.log(0.2e-3), n)), rng.uniform(0.2, 1.0, n)))
    g = synth.centred_grid(8, 8, 16, 0.1e-3)      # only its size is used: M = 1024
    w = synth.Workload("free-spread", g, synth.cap_sensors(8, 200e-3, 120.0), 8192, free=free)
    rel, y, yo = _check(w)
    assert np.abs(yo).max() > 0
