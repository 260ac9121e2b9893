"""Voxelisation (Eq. 2 sampled on a grid): CUDA path against the FP64 oracle, relative L2 1e-4."""
import numpy as np
import pytest
import torch

import oracle
from gpair_testutil import device_inputs, oracle_gaussians, rel_l2
from paper_2602_03893_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def _gpu_vox(w, og: synth.Grid, k):
    gs, _ = device_inputs(w)
    vol = torch.full((og.nz, og.ny, og.nx), float("nan"), device="cuda")
    _lib.gpair_voxelize(gs, _lib.Grid(og.nx, og.ny, og.nz, og.ox, og.oy, og.oz, og.h, og.sigma), k, vol)
    torch.cuda.synchronize()
    return vol.cpu().numpy()


def _ora_vox(w, og, k):
    return oracle.voxelize(oracle_gaussians(w), k, og.nx, og.ny, og.nz, og.ox, og.oy, og.oz, og.h)


@pytest.mark.parametrize("k", [3.0, 2.0])
def test_lattice_tiny(k):
    w = synth.tiny(1)
    v = _gpu_vox(w, w.grid, k)
    assert rel_l2(v, _ora_vox(w, w.grid, k)) < 1e-4


def test_lattice_mid():
    w = synth.mid(2)
    v = _gpu_vox(w, w.grid, 3.0)
    assert rel_l2(v, _ora_vox(w, w.grid, 3.0)) < 1e-4


def test_lattice_ragged_dims():
    g = synth.centred_grid(13, 7, 5, 0.1e-3)
    A = np.random.default_rng(1).uniform(0, 1, g.M).astype(np.float32)
    w = synth.Workload("ragged", g, synth.cap_sensors(1, 5e-3, 10.0), 16, A=A)
    assert rel_l2(_gpu_vox(w, g, 3.0), _ora_vox(w, g, 3.0)) < 1e-4


@pytest.mark.parametrize("k", [1.5, 4.2, 5.5, 6.0, 7.5])
def test_lattice_tap_counts_ragged(k):
    """Tap counts 1, 4, 5 and 6 a side (the fused three-axis kernel) and 7 (the separate passes)
    on a lattice whose sides are not multiples of the fused kernel's 32 x 8 x 16 block."""
    g = synth.centred_grid(37, 19, 21, 0.1e-3)
    A = np.random.default_rng(4).uniform(0, 1, g.M).astype(np.float32)
    w = synth.Workload("ragged-taps", g, synth.cap_sensors(1, 5e-3, 10.0), 16, A=A)
    assert rel_l2(_gpu_vox(w, g, k), _ora_vox(w, g, k)) < 1e-4


def test_free_gaussians_scatter_path():
    g = synth.centred_grid(24, 20, 16, 0.1e-3)
    free = synth.free_gaussians(g, 3, A=np.random.default_rng(2).uniform(0, 1, g.M))
    w = synth.Workload("free", g, synth.cap_sensors(1, 5e-3, 10.0), 16, free=free)
    og = synth.centred_grid(30, 26, 20, 0.08e-3)
    assert rel_l2(_gpu_vox(w, og, 3.0), _ora_vox(w, og, 3.0)) < 1e-4


def test_grid_gaussians_onto_other_grid():
    w = synth.tiny(1)
    og = synth.centred_grid(20, 18, 22, 0.15e-3)
    assert rel_l2(_gpu_vox(w, og, 3.0), _ora_vox(w, og, 3.0)) < 1e-4


def test_lattice_paper_scale_sampled_crops():
    """The benchmark's call (256 x 256 x 128 Gaussians onto their own lattice, k = 3: three
    separable passes with 4-output runs and compile-time taps) against the oracle on 14 crops of
    6 x 6 x 6 voxels, including faces, edges and corners of the volume.  Each crop's oracle sum
    takes every Gaussian within k sigma of it (a lattice margin of 4 nodes at sigma = h)."""
    w = synth.paper_scale(3)
    g = w.grid
    A = (np.random.default_rng(31).uniform(0.0, 1.0, g.M) ** 2).astype(np.float32)
    ww = synth.Workload(w.name, g, w.sensors[:1], 16, A=A)
    v = _gpu_vox(ww, g, 3.0)
    rng = np.random.default_rng(32)
    C, R = 6, 4
    starts = [(0, 0, 0), (g.nx - C, g.ny - C, g.nz - C), (0, g.ny - C, 0), (g.nx - C, 0, g.nz // 2),
              (g.nx // 2, 0, 0), (0, g.ny // 2, g.nz - C)]
    starts += [tuple(int(rng.integers(0, n - C + 1)) for n in (g.nx, g.ny, g.nz)) for _ in range(8)]
    A3 = A.reshape(g.nz, g.ny, g.nx)
    for (x0, y0, z0) in starts:
        xa, ya, za = max(0, x0 - R), max(0, y0 - R), max(0, z0 - R)
        xb, yb, zb = min(g.nx, x0 + C + R), min(g.ny, y0 + C + R), min(g.nz, z0 + C + R)
        # the crop's Gaussians and voxels share one lattice whose origin is 0 (voxelization depends
        # on differences only), so that offsets of exactly k sigma stay exact ties, as on the full
        # lattice; the crop's interior then has every Gaussian that reaches it
        nx, ny, nz = xb - xa, yb - ya, zb - za
        Gs = oracle.gaussians_from_grid(nx, ny, nz, 0.0, 0.0, 0.0, g.h, g.sigma,
                                        np.ascontiguousarray(A3[za:zb, ya:yb, xa:xb]).reshape(-1))
        full = oracle.voxelize(Gs, 3.0, nx, ny, nz, 0.0, 0.0, 0.0, g.h)
        ref = full[z0 - za:z0 - za + C, y0 - ya:y0 - ya + C, x0 - xa:x0 - xa + C]
        got = v[z0:z0 + C, y0:y0 + C, x0:x0 + C]
        assert rel_l2(got, ref) < 1e-4, (x0, y0, z0, rel_l2(got, ref))
