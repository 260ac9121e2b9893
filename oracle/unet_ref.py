"""FP64 CPU reference of the warm-start U-Net (test infrastructure only; used by tests/).

Plain torch.nn.functional on CPU in float64: 3x3x3 convolutions with zero padding 1, ReLU,
2x2x2 average pooling, nearest x2 upsampling, channel concatenation (upsampled first, then the
skip), and a 1x1x1 output convolution -- the same architecture the CUDA path implements,
evaluated in channels-first layout with torch autograd for the gradients.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

ORDER = ("e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "b4a", "b4b", "d3a", "d3b", "d2a", "d2b", "d1a", "d1b", "out")


def to_weight(w_cl: torch.Tensor, taps: int) -> torch.Tensor:
    """[Cout][taps][Cin] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) -> conv3d weight [Cout][Cin][kz][ky][kx]."""
    co, t, ci = w_cl.shape
    k = 3 if taps == 27 else 1
    return w_cl.reshape(co, k, k, k, ci).permute(0, 4, 1, 2, 3).contiguous()


def conv(x, w_cl, b, taps, relu):
    y = F.conv3d(x, to_weight(w_cl, taps), b, padding=1 if taps == 27 else 0)
    return F.relu(y) if relu else y


def unet_forward(x0: torch.Tensor, W: dict, B: dict) -> torch.Tensor:
    """x0: [1, 16, D, H, W] float64 (channels-first); W[name]: [Cout][taps][Cin]; returns [1, 16, D, H, W]."""
    T = lambda n: 1 if n == "out" else 27
    c = lambda n, x, relu=True: conv(x, W[n], B[n], T(n), relu)
    e1 = c("e1b", c("e1a", x0))
    e2 = c("e2b", c("e2a", F.avg_pool3d(e1, 2)))
    e3 = c("e3b", c("e3a", F.avg_pool3d(e2, 2)))
    b4 = c("b4b", c("b4a", F.avg_pool3d(e3, 2)))
    up = lambda x: F.interpolate(x, scale_factor=2, mode="nearest")
    d3 = c("d3b", c("d3a", torch.cat([up(b4), e3], 1)))
    d2 = c("d2b", c("d2a", torch.cat([up(d3), e2], 1)))
    d1 = c("d1b", c("d1a", torch.cat([up(d2), e1], 1)))
    return c("out", d1, relu=False)
