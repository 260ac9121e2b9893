"""Shared helpers for the parity tests: move a synthetic workload to the device (CUDA path)
and describe the same inputs to the oracle.  No operator arithmetic lives here."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2602_03893_gb300 import synth

# Window-decision tolerance: pairs whose |d| lies within TAU of k*sigma may be decided either way
# by an FP32 implementation (its phase error is ~1e-10 m), so the oracle reports their weight.
TAU = 4e-9


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_gaussians(w: synth.Workload, A=None) -> oracle.Gaussians:
    if w.free is not None:
        cx, cy, cz, sg, A0 = w.free
        return oracle.gaussians_from_soa(cx, cy, cz, sg, A0 if A is None else A)
    g = w.grid
    return oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, w.A if A is None else A)


def device_inputs(w: synth.Workload, A=None, k=None):
    """(Gaussians, SensorArray) on cuda:0 for the C ABI."""
    import torch
    from paper_2602_03893_gb300 import _lib

    dev = torch.device("cuda")
    if w.free is not None:
        cx, cy, cz, sg, A0 = w.free
        t = lambda q: torch.as_tensor(np.ascontiguousarray(q, dtype=np.float32), device=dev)
        gs = _lib.Gaussians(A=t(A0 if A is None else A), cx=t(cx), cy=t(cy), cz=t(cz), sigma=t(sg))
    else:
        g = w.grid
        AA = w.A if A is None else A
        gs = _lib.Gaussians(A=torch.as_tensor(np.ascontiguousarray(AA, dtype=np.float32), device=dev),
                            grid=_lib.Grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma))
    arr = _lib.SensorArray(xyz=torch.as_tensor(np.ascontiguousarray(w.sensors, dtype=np.float32), device=dev),
                           sound_speed=w.v, fs=w.fs, n_samples=w.Nt, t0=w.t0, window_k=w.k if k is None else k)
    return gs, arr


def gpu_forward(w: synth.Workload, A=None, k=None) -> np.ndarray:
    import torch
    from paper_2602_03893_gb300 import _lib

    gs, arr = device_inputs(w, A, k)
    y = torch.full((w.Nd, w.Nt), float("nan"), device="cuda", dtype=torch.float32)
    _lib.gpair_forward(gs, arr, y)
    torch.cuda.synchronize()
    assert _lib.gpair_last_device_status() == 0
    return y.cpu().numpy()


def gpu_adjoint(w: synth.Workload, delta: np.ndarray, full: bool, A=None, k=None):
    import torch
    from paper_2602_03893_gb300 import _lib

    gs, arr = device_inputs(w, A, k)
    M = gs.M
    d = torch.as_tensor(np.ascontiguousarray(delta, dtype=np.float32), device="cuda")
    gA = torch.full((M,), float("nan"), device="cuda")
    gc = torch.full((3, M), float("nan"), device="cuda") if full else None
    gsg = torch.full((M,), float("nan"), device="cuda") if full else None
    _lib.gpair_adjoint(gs, arr, d, gA, gc, gsg)
    torch.cuda.synchronize()
    out = {"A": gA.cpu().numpy()}
    if full:
        out["c"] = gc.cpu().numpy()
        out["sigma"] = gsg.cpu().numpy()
    return out


def assert_signal_parity(y_gpu, y_ora, amb, tol=1e-5):
    """Relative L2 within tol, allowing the weight of window-ambiguous terms."""
    err = np.linalg.norm(np.asarray(y_gpu, np.float64) - y_ora)
    bound = tol * np.linalg.norm(y_ora) + (np.linalg.norm(amb) if amb is not None else 0.0)
    assert np.all(np.isfinite(y_gpu))
    assert err <= bound, f"|err| {err:.3e} > bound {bound:.3e} (rel {err / max(np.linalg.norm(y_ora), 1e-300):.3e})"
    return err / max(np.linalg.norm(y_ora), 1e-300)


def edge_workload(sigma_scale):
    """Tiny geometry with sigma = sigma_scale * h: 2 k sigma / Delta = 32 sigma_scale, so the
    window's edge position E = floor(2 k sigma / Delta) is inside for a fraction 0.32 (1.01) or
    0.64 (1.02) of the pairs."""
    g = synth.centred_grid(16, 16, 16, 0.2e-3, sigma=0.2e-3 * sigma_scale)
    A = np.random.default_rng(11).uniform(0.0, 1.0, g.M).astype(np.float32)
    return synth.Workload("edge", g, synth.cap_sensors(128, 20e-3, 180.0), 1024, A=A)
