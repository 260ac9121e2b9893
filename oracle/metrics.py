"""FP64 oracle of the image metrics the paper tabulates for reconstructions (Results, Table 1:
PSNR, SSIM and MSE on the 3-D volume and on its maximum amplitude projection along z).

TEST INFRASTRUCTURE ONLY: loaded by tests/ (and nothing in the product package).

The paper names the metrics without formulas; the readings taken (the common definitions):
  - Z-MAP: the maximum over z of the volume, an (ny, nx) image;
  - MSE: mean squared difference; PSNR = 10 log10(data_range^2 / MSE);
  - SSIM (Wang et al., 2004): local means, variances and covariance over a uniform window of
    `win` samples per axis (7), variances and covariance with the sample normalisation
    N / (N - 1), C1 = (0.01 data_range)^2, C2 = (0.03 data_range)^2,
        s = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
    averaged over the positions whose whole window lies inside the image (2-D or 3-D).
Inputs are float64 arrays of equal shape.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def zmap(vol):
    """Maximum amplitude projection along z of a (nz, ny, nx) volume."""
    return np.asarray(vol, dtype=np.float64).max(axis=0)


def mse(x, ref):
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    return float(np.mean((x - ref) ** 2))


def psnr(x, ref, data_range=1.0):
    return float(10.0 * np.log10(data_range ** 2 / mse(x, ref)))


def ssim(x, ref, win=7, data_range=1.0, K1=0.01, K2=0.03):
    x, y = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    N = win ** x.ndim
    f = lambda a: ndimage.uniform_filter(a, size=win, mode="reflect")
    mx, my = f(x), f(y)
    cov = N / (N - 1.0)
    sxx = cov * (f(x * x) - mx * mx)
    syy = cov * (f(y * y) - my * my)
    sxy = cov * (f(x * y) - mx * my)
    C1, C2 = (K1 * data_range) ** 2, (K2 * data_range) ** 2
    s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    p = (win - 1) // 2
    inner = tuple(slice(p, n - p) for n in x.shape)
    return float(s[inner].mean())
