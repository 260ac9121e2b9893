"""FP64 CPU reference of the warm-start U-Net (test infrastructure only; used by tests/).

The network (the learned warm start of the benchmark's fifth configuration: four levels with
16, 32, 64 and 128 channels, one channel in and one out): two 3x3x3 convolutions with zero
padding 1 and ReLU per level, 2x2x2 average pooling down, nearest x2 upsampling and channel
concatenation (upsampled first, then the skip) up, and a 1x1x1 output convolution.  The input
channel is stored padded to 16 channels (15 zero) and the output convolution computes 16
channels of which channel 0 is the prediction; both paddings are exact.

Two evaluations of the same definition live here:

* `conv`, `pool`, `up`, `unet_forward`: torch.nn.functional on CPU in float64 (channels-first),
  differentiable with torch autograd -- what the GPU tests compare against.  With
  `bf16_storage=True` every stored activation (convolution outputs, pooled, upsampled and
  concatenated tensors) is rounded to BF16, and so is the gradient that reaches it in the
  backward pass (`RoundBF16`): the storage precision the configuration fixes for weights and
  activations, while all arithmetic stays FP64.
* `conv_loops`, `pool_loops`, `up_loops`, `unet_forward_loops`: the same operations written out
  as sums over taps, window cells and channels on numpy arrays, with `bf16_round_loops` as an
  independent round-to-nearest-even on the float32 bit pattern.  They pin the torch evaluation
  (tests/test_oracle_pins.py) and are slow; tiny volumes only.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

ORDER = ("e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "b4a", "b4b", "d3a", "d3b", "d2a", "d2b", "d1a", "d1b", "out")

# The architecture: channels per level, the channel widths as stored, and every convolution as
# (name, input channels, output channels, taps, ReLU).
LEVEL_CHANNELS = (16, 32, 64, 128)
IN_CHANNELS, OUT_CHANNELS = 1, 1
IN_STORED, OUT_STORED = 16, 16


def architecture():
    c1, c2, c3, c4 = LEVEL_CHANNELS
    return (("e1a", IN_STORED, c1, 27, True), ("e1b", c1, c1, 27, True),
            ("e2a", c1, c2, 27, True), ("e2b", c2, c2, 27, True),
            ("e3a", c2, c3, 27, True), ("e3b", c3, c3, 27, True),
            ("b4a", c3, c4, 27, True), ("b4b", c4, c4, 27, True),
            ("d3a", c4 + c3, c3, 27, True), ("d3b", c3, c3, 27, True),
            ("d2a", c3 + c2, c2, 27, True), ("d2b", c2, c2, 27, True),
            ("d1a", c2 + c1, c1, 27, True), ("d1b", c1, c1, 27, True),
            ("out", c1, OUT_STORED, 1, False))


def to_weight(w_cl: torch.Tensor, taps: int) -> torch.Tensor:
    """[Cout][taps][Cin] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)) -> conv3d weight [Cout][Cin][kz][ky][kx]."""
    co, t, ci = w_cl.shape
    k = 3 if taps == 27 else 1
    return w_cl.reshape(co, k, k, k, ci).permute(0, 4, 1, 2, 3).contiguous()


class RoundBF16(torch.autograd.Function):
    """Identity in exact arithmetic; rounds the stored value to BF16 going forward and the
    gradient that reaches the stored value going backward (float64 in, float64 out)."""

    @staticmethod
    def forward(ctx, x):
        return x.to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(torch.float64)


def _store(x, bf16):
    return RoundBF16.apply(x) if bf16 else x


def conv(x, w_cl, b, taps, relu):
    y = F.conv3d(x, to_weight(w_cl, taps), b, padding=1 if taps == 27 else 0)
    return F.relu(y) if relu else y


def pool(x):
    return F.avg_pool3d(x, 2)


def up(x):
    return F.interpolate(x, scale_factor=2, mode="nearest")


def unet_forward(x0: torch.Tensor, W: dict, B: dict, bf16_storage: bool = False) -> torch.Tensor:
    """x0: [1, 16, D, H, W] float64 (channels-first); W[name]: [Cout][taps][Cin]; returns [1, 16, D, H, W].
    bf16_storage: round every stored activation (and the gradient reaching it) to BF16."""
    T = {n: taps for n, _, _, taps, _ in architecture()}
    R = {n: relu for n, _, _, _, relu in architecture()}
    s = lambda x: _store(x, bf16_storage)
    c = lambda n, x: s(conv(x, W[n], B[n], T[n], R[n]))
    x0 = s(x0)
    e1 = c("e1b", c("e1a", x0))
    e2 = c("e2b", c("e2a", s(pool(e1))))
    e3 = c("e3b", c("e3a", s(pool(e2))))
    b4 = c("b4b", c("b4a", s(pool(e3))))
    d3 = c("d3b", c("d3a", s(torch.cat([s(up(b4)), e3], 1))))
    d2 = c("d2b", c("d2a", s(torch.cat([s(up(d3)), e2], 1))))
    d1 = c("d1b", c("d1a", s(torch.cat([s(up(d2)), e1], 1))))
    return c("out", d1)


# ---------------------------------------------------------------- plain loops (numpy, float64)

def bf16_round_loops(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (8 significant bits), nearest with ties to even, through float32: keep the
    upper 16 bits of the float32 pattern after adding 0x7FFF plus the lowest kept bit."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + keep_lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def conv_loops(x: np.ndarray, w_cl: np.ndarray, b: np.ndarray, taps: int, relu: bool) -> np.ndarray:
    """x [Cin][D][H][W]; w_cl [Cout][taps][Cin]; b [Cout].
    y[o, z, y, x] = b[o] + sum over taps (dz, dy, dx) and input channels i of
    w[o, tap, i] * x[i, z + dz, y + dy, x + dx], with x = 0 outside the volume."""
    ci, D, H, Wd = x.shape
    co = w_cl.shape[0]
    r = 1 if taps == 27 else 0
    y = np.empty((co, D, H, Wd))
    for z in range(D):
        for yy in range(H):
            for xx in range(Wd):
                acc = np.array(b, dtype=np.float64)        # all output channels of this voxel
                tap = 0
                for dz in range(-r, r + 1):
                    for dy in range(-r, r + 1):
                        for dx in range(-r, r + 1):
                            zz, y2, x2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < Wd:
                                acc = acc + w_cl[:, tap, :] @ x[:, zz, y2, x2]   # sum over input channels
                            tap += 1
                y[:, z, yy, xx] = np.maximum(acc, 0.0) if relu else acc
    return y


def pool_loops(x: np.ndarray) -> np.ndarray:
    """Mean of each 2 x 2 x 2 cell."""
    C, D, H, Wd = x.shape
    y = np.zeros((C, D // 2, H // 2, Wd // 2))
    for c in range(C):
        for z in range(D // 2):
            for yy in range(H // 2):
                for xx in range(Wd // 2):
                    s = 0.0
                    for a in range(2):
                        for bb in range(2):
                            for cc in range(2):
                                s += x[c, 2 * z + a, 2 * yy + bb, 2 * xx + cc]
                    y[c, z, yy, xx] = s / 8.0
    return y


def up_loops(x: np.ndarray) -> np.ndarray:
    """Nearest-neighbour x2: output voxel (z, y, x) copies input voxel (z // 2, y // 2, x // 2)."""
    C, D, H, Wd = x.shape
    y = np.zeros((C, 2 * D, 2 * H, 2 * Wd))
    for z in range(2 * D):
        for yy in range(2 * H):
            for xx in range(2 * Wd):
                y[:, z, yy, xx] = x[:, z // 2, yy // 2, xx // 2]
    return y


def unet_forward_loops(x0: np.ndarray, W: dict, B: dict, bf16_storage: bool = False) -> np.ndarray:
    """The network of `architecture()` on x0 [16][D][H][W] with the loop operations above."""
    spec = {n: (taps, relu) for n, _, _, taps, relu in architecture()}
    s = (lambda x: bf16_round_loops(x)) if bf16_storage else (lambda x: x)
    c = lambda n, x: s(conv_loops(x, W[n], B[n], *spec[n]))
    x0 = s(x0)
    e1 = c("e1b", c("e1a", x0))
    e2 = c("e2b", c("e2a", s(pool_loops(e1))))
    e3 = c("e3b", c("e3a", s(pool_loops(e2))))
    b4 = c("b4b", c("b4a", s(pool_loops(e3))))
    d3 = c("d3b", c("d3a", s(np.concatenate([s(up_loops(b4)), e3], 0))))
    d2 = c("d2b", c("d2a", s(np.concatenate([s(up_loops(d3)), e2], 0))))
    d1 = c("d1b", c("d1a", s(np.concatenate([s(up_loops(d2)), e1], 0))))
    return c("out", d1)
