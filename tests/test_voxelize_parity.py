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
