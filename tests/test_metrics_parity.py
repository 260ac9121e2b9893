"""Image metrics of reconstructions (Results, Table 1: PSNR, SSIM, MSE on the volume and on its
Z-MAP): gpair_zmap and gpair_image_metrics against the FP64 oracle.  The projection is exact
(a maximum); MSE and PSNR to 1e-6 relative (FP32 differences, FP64 sums); SSIM to 1e-5 absolute
(FP32 box sums of x, y, x^2, y^2, xy; the variance differences they form are small against C2)."""
import numpy as np
import pytest
import torch

from oracle import metrics
from paper_2602_03893_gb300 import _lib

pytestmark = pytest.mark.gpu


# windows up to 15 take the fused pass (ragged column tiles of 32 x 8 and z chunks of 16 below);
# 17 takes the per-axis passes through device memory
@pytest.mark.parametrize("dims,win", [((20, 24, 28), 7), ((1, 50, 61), 7), ((9, 11, 13), 3), ((7, 7, 7), 7),
                                      ((37, 45, 70), 7), ((1, 33, 65), 15), ((17, 18, 40), 15), ((19, 20, 21), 17)])
def test_metrics_against_oracle(dims, win):
    rng = np.random.default_rng(sum(dims))
    ref = rng.uniform(0, 1, dims).astype(np.float32)
    x = np.clip(ref + rng.normal(0, 0.1, dims), 0, 1).astype(np.float32)
    got = _lib.gpair_image_metrics(torch.as_tensor(x, device="cuda"), torch.as_tensor(ref, device="cuda"), dims, win)
    xd, rd = x.astype(np.float64), ref.astype(np.float64)
    sq = (lambda a: a[0]) if dims[0] == 1 else (lambda a: a)
    exp_mse = metrics.mse(xd, rd)
    assert abs(got["mse"] - exp_mse) <= 1e-6 * exp_mse
    assert abs(got["psnr"] - metrics.psnr(xd, rd)) <= 1e-5
    assert abs(got["ssim"] - metrics.ssim(sq(xd), sq(rd), win=win)) <= 1e-5


def test_zmap_is_exact_and_feeds_the_2d_metrics():
    dims = (17, 40, 48)
    rng = np.random.default_rng(3)
    vol = rng.uniform(0, 1, dims).astype(np.float32)
    ref = rng.uniform(0, 1, dims).astype(np.float32)
    m = _lib.gpair_zmap(torch.as_tensor(vol, device="cuda"), dims).cpu().numpy()
    assert np.array_equal(m, metrics.zmap(vol).astype(np.float32))
    mr = metrics.zmap(ref).astype(np.float32)
    got = _lib.gpair_image_metrics(torch.as_tensor(m, device="cuda"), torch.as_tensor(mr, device="cuda"),
                                   (1, dims[1], dims[2]))
    assert abs(got["ssim"] - metrics.ssim(m.astype(np.float64), mr.astype(np.float64))) <= 1e-5


def test_identical_images_and_rejections():
    x = torch.rand((8, 9, 10), device="cuda")
    got = _lib.gpair_image_metrics(x, x.clone(), (8, 9, 10), 7)
    assert got["mse"] == 0.0 and abs(got["ssim"] - 1.0) < 1e-6
    with pytest.raises(_lib.GpairError):
        _lib.gpair_image_metrics(x, x, (8, 9, 10), 4)            # even window
    with pytest.raises(_lib.GpairError):
        _lib.gpair_image_metrics(x[:5].contiguous(), x[:5].contiguous(), (5, 9, 10), 7)   # z shorter than the window


def test_paper_scale_volume():
    """The benchmark's 256 x 256 x 128 volume (2048 column-chunk items over the persistent CTAs)."""
    dims = (128, 256, 256)
    rng = np.random.default_rng(41)
    ref = rng.uniform(0, 1, dims).astype(np.float32)
    x = np.clip(ref + rng.normal(0, 0.05, dims), 0, 1).astype(np.float32)
    got = _lib.gpair_image_metrics(torch.as_tensor(x, device="cuda"), torch.as_tensor(ref, device="cuda"), dims, 7)
    xd, rd = x.astype(np.float64), ref.astype(np.float64)
    exp_mse = metrics.mse(xd, rd)
    assert abs(got["mse"] - exp_mse) <= 1e-6 * exp_mse
    assert abs(got["ssim"] - metrics.ssim(xd, rd, win=7)) <= 1e-5
