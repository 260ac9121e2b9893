"""Learned warm start: a 3-D U-Net that maps the adjoint back-projection A^T b of measured signals
to initial Gaussian amplitudes (the paper's Discussion: the ImageReconstructor as an initialiser,
and the operators as a differentiable physics layer in learned pipelines).

Four levels with 16, 32, 64 and 128 channels; two 3x3x3 convolutions + ReLU per level, 2x2x2
average pooling down, nearest x2 upsampling and skip concatenation up, and a 1x1x1 output
convolution.  Weights and activations are bf16, every kernel accumulates in FP32, weights keep
FP32 master copies for Adam.  Every step runs in libgpair's kernels (include/gpair_unet.h);
torch tensors only hold device memory.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

P = ctypes.c_void_p
CIN_PAD = 16     # the single input channel is stored as 16 (fragment width); 15 are zero
COUT_PAD = 16    # the output convolution computes 16 channels; channel 0 is the prediction

_bound = False


def _unet_lib():
    global _bound
    lib = _lib.load()
    if not _bound:
        i32, i64, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_float
        lib.gpair_conv3d_fwd.argtypes = [P, i32, i32, i32, i32, P, P, i32, i32, i32, P, P]
        lib.gpair_conv3d_dgrad.argtypes = [P, i32, i32, i32, i32, P, i32, i32, P, P, P]
        lib.gpair_conv3d_wgrad.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P, P, P]
        lib.gpair_relu_bwd.argtypes = [P, P, i64, P]
        lib.gpair_pool2_fwd.argtypes = [P, i32, i32, i32, i32, P, P]
        lib.gpair_pool2_bwd.argtypes = [P, i32, i32, i32, i32, P, P]
        lib.gpair_up2_fwd.argtypes = [P, i32, i32, i32, i32, P, P]
        lib.gpair_up2_bwd.argtypes = [P, i32, i32, i32, i32, P, P]
        lib.gpair_concat_fwd.argtypes = [P, i32, P, i32, i64, P, P]
        lib.gpair_concat_bwd.argtypes = [P, i32, i32, i64, P, P, P]
        lib.gpair_add_bf16.argtypes = [P, P, P, i64, P]
        lib.gpair_pack_input.argtypes = [P, f32, i64, i32, P, P]
        lib.gpair_unpack_output.argtypes = [P, i64, i32, f32, i32, P, P]
        lib.gpair_mse_loss.argtypes = [P, P, i64, i32, P, P, P]
        lib.gpair_adam_bf16.argtypes = [P, P, P, P, P, i64, f32, f32, f32, f32, i32, P]
        lib.gpair_unet_tensor_path.argtypes = [i32]
        lib.gpair_unet_tensor_path.restype = i32
        lib.gpair_unet_tc_status.argtypes = []
        lib.gpair_unet_tc_status.restype = i32
        _bound = True
    return lib


def _p(t):
    return None if t is None else t.data_ptr()


def _s():
    return P(torch.cuda.current_stream().cuda_stream)


def _ck(name, code):
    if code != 0:
        raise _lib.GpairError(name, code)


# ---------------------------------------------------------------- thin wrappers (same names)

def gpair_unet_tensor_path(mode: int = -1) -> int:
    """1 (default): the tcgen05 tensor-core convolution for every eligible shape, mma.sync for the
    others; 2: tcgen05 only; 0: mma.sync only; other values query.  Returns the mode in force."""
    return int(_unet_lib().gpair_unet_tensor_path(int(mode)))


def gpair_unet_tc_status() -> int:
    return int(_unet_lib().gpair_unet_tc_status())


def gpair_conv3d_fwd(x, dims, Cin, w, b, Cout, taps, relu, out):
    D, H, W = dims
    _ck("gpair_conv3d_fwd", _unet_lib().gpair_conv3d_fwd(_p(x), D, H, W, Cin, _p(w), _p(b), Cout, taps, int(relu),
                                                         _p(out), _s()))
    return out


def gpair_conv3d_dgrad(dout, dims, Cout, w, Cin, taps, wt_scratch, din):
    D, H, W = dims
    _ck("gpair_conv3d_dgrad", _unet_lib().gpair_conv3d_dgrad(_p(dout), D, H, W, Cout, _p(w), Cin, taps,
                                                             _p(wt_scratch), _p(din), _s()))
    return din


def gpair_conv3d_wgrad(x, dout, dims, Cin, Cout, taps, dw, db):
    D, H, W = dims
    _ck("gpair_conv3d_wgrad", _unet_lib().gpair_conv3d_wgrad(_p(x), _p(dout), D, H, W, Cin, Cout, taps, _p(dw),
                                                             _p(db), _s()))


def gpair_relu_bwd(act, g):
    _ck("gpair_relu_bwd", _unet_lib().gpair_relu_bwd(_p(act), _p(g), g.numel(), _s()))


def gpair_pool2_fwd(x, dims, C, out):
    _ck("gpair_pool2_fwd", _unet_lib().gpair_pool2_fwd(_p(x), *dims, C, _p(out), _s()))


def gpair_pool2_bwd(dout, dims, C, din):
    _ck("gpair_pool2_bwd", _unet_lib().gpair_pool2_bwd(_p(dout), *dims, C, _p(din), _s()))


def gpair_up2_fwd(x, dims, C, out):
    _ck("gpair_up2_fwd", _unet_lib().gpair_up2_fwd(_p(x), *dims, C, _p(out), _s()))


def gpair_up2_bwd(dout, dims, C, din):
    _ck("gpair_up2_bwd", _unet_lib().gpair_up2_bwd(_p(dout), *dims, C, _p(din), _s()))


def gpair_concat_fwd(a, Ca, b, Cb, nv, out):
    _ck("gpair_concat_fwd", _unet_lib().gpair_concat_fwd(_p(a), Ca, _p(b), Cb, nv, _p(out), _s()))


def gpair_concat_bwd(dout, Ca, Cb, nv, da, db):
    _ck("gpair_concat_bwd", _unet_lib().gpair_concat_bwd(_p(dout), Ca, Cb, nv, _p(da), _p(db), _s()))


def gpair_add_bf16(a, b, out):
    _ck("gpair_add_bf16", _unet_lib().gpair_add_bf16(_p(a), _p(b), _p(out), out.numel(), _s()))


def gpair_pack_input(x, scale, nv, C, out):
    _ck("gpair_pack_input", _unet_lib().gpair_pack_input(_p(x), float(scale), nv, C, _p(out), _s()))


def gpair_unpack_output(x, nv, C, scale, relu, out):
    _ck("gpair_unpack_output", _unet_lib().gpair_unpack_output(_p(x), nv, C, float(scale), int(relu), _p(out), _s()))


def gpair_mse_loss(pred, target, nv, C, dpred, loss):
    _ck("gpair_mse_loss", _unet_lib().gpair_mse_loss(_p(pred), _p(target), nv, C, _p(dpred), _p(loss), _s()))


def gpair_adam_bf16(w, g, m, v, wb, lr, b1, b2, eps, t):
    _ck("gpair_adam_bf16", _unet_lib().gpair_adam_bf16(_p(w), _p(g), _p(m), _p(v), _p(wb), w.numel(), float(lr),
                                                       float(b1), float(b2), float(eps), int(t), _s()))


# ---------------------------------------------------------------- network

@dataclass
class Conv:
    cin: int
    cout: int
    taps: int
    relu: bool


def layer_specs(ch=(16, 32, 64, 128)) -> dict:
    """Every convolution of the network: name -> Conv(input channels, output channels, taps, ReLU)."""
    c1, c2, c3, c4 = ch
    return {
        "e1a": Conv(CIN_PAD, c1, 27, True), "e1b": Conv(c1, c1, 27, True),
        "e2a": Conv(c1, c2, 27, True), "e2b": Conv(c2, c2, 27, True),
        "e3a": Conv(c2, c3, 27, True), "e3b": Conv(c3, c3, 27, True),
        "b4a": Conv(c3, c4, 27, True), "b4b": Conv(c4, c4, 27, True),
        "d3a": Conv(c4 + c3, c3, 27, True), "d3b": Conv(c3, c3, 27, True),
        "d2a": Conv(c3 + c2, c2, 27, True), "d2b": Conv(c2, c2, 27, True),
        "d1a": Conv(c2 + c1, c1, 27, True), "d1b": Conv(c1, c1, 27, True),
        "out": Conv(c1, COUT_PAD, 1, False),
    }


def bf16(shape, dev):
    return torch.empty(shape, dtype=torch.bfloat16, device=dev)


class UNet3D:
    """The U-Net on a D x H x W volume (each divisible by 8)."""

    CH = (16, 32, 64, 128)

    def __init__(self, dims, device="cuda", seed=0):
        self.dims = tuple(int(d) for d in dims)
        assert all(d % 8 == 0 for d in self.dims), "U-Net volume sides must be divisible by 8"
        self.dev = torch.device(device)
        self.convs = layer_specs(self.CH)
        gen = torch.Generator(device="cpu").manual_seed(seed)
        self.w32, self.wbf, self.b32, self.bbf, self.gw, self.gb = {}, {}, {}, {}, {}, {}
        self.mw, self.vw, self.mb, self.vb = {}, {}, {}, {}
        for name, c in self.convs.items():
            fan_in = c.taps * (1 if name == "e1a" else c.cin)
            std = math.sqrt(2.0 / fan_in) if c.relu else math.sqrt(1.0 / fan_in)
            w = torch.randn((c.cout, c.taps, c.cin), generator=gen) * std
            if name == "e1a":
                w[:, :, 1:] = 0.0             # padding channels of the input
            if name == "out":
                w[1:] = 0.0                   # only channel 0 is used
            self.w32[name] = w.to(self.dev).contiguous()
            self.wbf[name] = self.w32[name].to(torch.bfloat16).contiguous()
            self.b32[name] = torch.zeros(c.cout, device=self.dev)
            self.bbf[name] = torch.zeros(c.cout, device=self.dev, dtype=torch.bfloat16)
            for d in (self.gw, self.mw, self.vw):
                d[name] = torch.zeros_like(self.w32[name])
            for d in (self.gb, self.mb, self.vb):
                d[name] = torch.zeros_like(self.b32[name])
        self.t = 0
        maxw = max(c.cout * c.taps * c.cin for c in self.convs.values())
        self.wt_scratch = bf16((maxw,), self.dev)
        self._alloc()

    def levels(self):
        D, H, W = self.dims
        return [(D >> q, H >> q, W >> q) for q in range(4)]

    def _alloc(self):
        L = self.levels()
        nv = [d[0] * d[1] * d[2] for d in L]
        c1, c2, c3, c4 = self.CH
        a = {}
        a["x"] = bf16((nv[0], CIN_PAD), self.dev)
        a["e1a"], a["e1b"] = bf16((nv[0], c1), self.dev), bf16((nv[0], c1), self.dev)
        a["p1"] = bf16((nv[1], c1), self.dev)
        a["e2a"], a["e2b"] = bf16((nv[1], c2), self.dev), bf16((nv[1], c2), self.dev)
        a["p2"] = bf16((nv[2], c2), self.dev)
        a["e3a"], a["e3b"] = bf16((nv[2], c3), self.dev), bf16((nv[2], c3), self.dev)
        a["p3"] = bf16((nv[3], c3), self.dev)
        a["b4a"], a["b4b"] = bf16((nv[3], c4), self.dev), bf16((nv[3], c4), self.dev)
        a["u3"] = bf16((nv[2], c4), self.dev)
        a["k3"] = bf16((nv[2], c4 + c3), self.dev)
        a["d3a"], a["d3b"] = bf16((nv[2], c3), self.dev), bf16((nv[2], c3), self.dev)
        a["u2"] = bf16((nv[1], c3), self.dev)
        a["k2"] = bf16((nv[1], c3 + c2), self.dev)
        a["d2a"], a["d2b"] = bf16((nv[1], c2), self.dev), bf16((nv[1], c2), self.dev)
        a["u1"] = bf16((nv[0], c2), self.dev)
        a["k1"] = bf16((nv[0], c2 + c1), self.dev)
        a["d1a"], a["d1b"] = bf16((nv[0], c1), self.dev), bf16((nv[0], c1), self.dev)
        a["out"] = bf16((nv[0], COUT_PAD), self.dev)
        self.act = a
        # gradient buffers (same shapes); reused across steps
        self.grad = {k: torch.empty_like(v) for k, v in a.items() if k != "x"}
        # pooled-path gradient of each encoder output before it is added to the skip gradient
        self.tmp = {0: bf16((nv[0], c1), self.dev), 1: bf16((nv[1], c2), self.dev), 2: bf16((nv[2], c3), self.dev)}
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.nv = nv

    # -------- forward / backward

    def _conv(self, name, x, dims, out):
        c = self.convs[name]
        gpair_conv3d_fwd(x, dims, c.cin, self.wbf[name], self.b32[name], c.cout, c.taps, c.relu, out)

    def forward(self, x_f32, in_scale=1.0):
        """x_f32: FP32 [nv] (A^T b on the grid).  Returns the bf16 output tensor [nv, 16]."""
        L, a = self.levels(), self.act
        c1, c2, c3, c4 = self.CH
        gpair_pack_input(x_f32, in_scale, self.nv[0], CIN_PAD, a["x"])
        self._conv("e1a", a["x"], L[0], a["e1a"])
        self._conv("e1b", a["e1a"], L[0], a["e1b"])
        gpair_pool2_fwd(a["e1b"], L[0], c1, a["p1"])
        self._conv("e2a", a["p1"], L[1], a["e2a"])
        self._conv("e2b", a["e2a"], L[1], a["e2b"])
        gpair_pool2_fwd(a["e2b"], L[1], c2, a["p2"])
        self._conv("e3a", a["p2"], L[2], a["e3a"])
        self._conv("e3b", a["e3a"], L[2], a["e3b"])
        gpair_pool2_fwd(a["e3b"], L[2], c3, a["p3"])
        self._conv("b4a", a["p3"], L[3], a["b4a"])
        self._conv("b4b", a["b4a"], L[3], a["b4b"])
        gpair_up2_fwd(a["b4b"], L[3], c4, a["u3"])
        gpair_concat_fwd(a["u3"], c4, a["e3b"], c3, self.nv[2], a["k3"])
        self._conv("d3a", a["k3"], L[2], a["d3a"])
        self._conv("d3b", a["d3a"], L[2], a["d3b"])
        gpair_up2_fwd(a["d3b"], L[2], c3, a["u2"])
        gpair_concat_fwd(a["u2"], c3, a["e2b"], c2, self.nv[1], a["k2"])
        self._conv("d2a", a["k2"], L[1], a["d2a"])
        self._conv("d2b", a["d2a"], L[1], a["d2b"])
        gpair_up2_fwd(a["d2b"], L[1], c2, a["u1"])
        gpair_concat_fwd(a["u1"], c2, a["e1b"], c1, self.nv[0], a["k1"])
        self._conv("d1a", a["k1"], L[0], a["d1a"])
        self._conv("d1b", a["d1a"], L[0], a["d1b"])
        self._conv("out", a["d1b"], L[0], a["out"])
        return a["out"]

    def _back_conv(self, name, x_in, dims, g_out, g_in, act_out=None):
        """g_out: gradient w.r.t. the conv's activation output (ReLU applied through act_out);
        accumulates dW, db; writes g_in = gradient w.r.t. the conv input (if g_in is not None)."""
        c = self.convs[name]
        if c.relu:
            gpair_relu_bwd(act_out, g_out)
        gpair_conv3d_wgrad(x_in, g_out, dims, c.cin, c.cout, c.taps, self.gw[name], self.gb[name])
        if g_in is not None:
            gpair_conv3d_dgrad(g_out, dims, c.cout, self.wbf[name], c.cin, c.taps, self.wt_scratch, g_in)

    def backward(self, g_out):
        """g_out: bf16 [nv, 16] gradient of the loss w.r.t. the output tensor."""
        L, a, g = self.levels(), self.act, self.grad
        c1, c2, c3, c4 = self.CH
        for d in (self.gw, self.gb):
            for t in d.values():
                t.zero_()
        self._back_conv("out", a["d1b"], L[0], g_out, g["d1b"])
        self._back_conv("d1b", a["d1a"], L[0], g["d1b"], g["d1a"], a["d1b"])
        self._back_conv("d1a", a["k1"], L[0], g["d1a"], g["k1"], a["d1a"])
        gpair_concat_bwd(g["k1"], c2, c1, self.nv[0], g["u1"], g["e1b"])        # g[e1b] = skip part
        gpair_up2_bwd(g["u1"], L[1], c2, g["d2b"])
        self._back_conv("d2b", a["d2a"], L[1], g["d2b"], g["d2a"], a["d2b"])
        self._back_conv("d2a", a["k2"], L[1], g["d2a"], g["k2"], a["d2a"])
        gpair_concat_bwd(g["k2"], c3, c2, self.nv[1], g["u2"], g["e2b"])
        gpair_up2_bwd(g["u2"], L[2], c3, g["d3b"])
        self._back_conv("d3b", a["d3a"], L[2], g["d3b"], g["d3a"], a["d3b"])
        self._back_conv("d3a", a["k3"], L[2], g["d3a"], g["k3"], a["d3a"])
        gpair_concat_bwd(g["k3"], c4, c3, self.nv[2], g["u3"], g["e3b"])
        gpair_up2_bwd(g["u3"], L[3], c4, g["b4b"])
        self._back_conv("b4b", a["b4a"], L[3], g["b4b"], g["b4a"], a["b4b"])
        self._back_conv("b4a", a["p3"], L[3], g["b4a"], g["p3"], a["b4a"])
        # e3b receives the skip gradient and the pooled path's gradient
        t = self.tmp[2]
        gpair_pool2_bwd(g["p3"], L[2], c3, t)
        gpair_add_bf16(g["e3b"], t, g["e3b"])
        self._back_conv("e3b", a["e3a"], L[2], g["e3b"], g["e3a"], a["e3b"])
        self._back_conv("e3a", a["p2"], L[2], g["e3a"], g["p2"], a["e3a"])
        t = self.tmp[1]
        gpair_pool2_bwd(g["p2"], L[1], c2, t)
        gpair_add_bf16(g["e2b"], t, g["e2b"])
        self._back_conv("e2b", a["e2a"], L[1], g["e2b"], g["e2a"], a["e2b"])
        self._back_conv("e2a", a["p1"], L[1], g["e2a"], g["p1"], a["e2a"])
        t = self.tmp[0]
        gpair_pool2_bwd(g["p1"], L[0], c1, t)
        gpair_add_bf16(g["e1b"], t, g["e1b"])
        self._back_conv("e1b", a["e1a"], L[0], g["e1b"], g["e1a"], a["e1b"])
        self._back_conv("e1a", a["x"], L[0], g["e1a"], None, a["e1a"])

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        for name in self.convs:
            gpair_adam_bf16(self.w32[name], self.gw[name], self.mw[name], self.vw[name], self.wbf[name], lr, b1, b2,
                            eps, self.t)
            gpair_adam_bf16(self.b32[name], self.gb[name], self.mb[name], self.vb[name], self.bbf[name], lr, b1, b2,
                            eps, self.t)

    def train_step(self, x_f32, target_f32, lr, in_scale=1.0):
        out = self.forward(x_f32, in_scale)
        self.loss.zero_()
        gpair_mse_loss(out, target_f32, self.nv[0], COUT_PAD, self.grad["out"], self.loss)
        self.backward(self.grad["out"])
        self.step(lr)
        return self.loss

    def predict(self, x_f32, in_scale=1.0, out_scale=1.0, relu=True):
        out = self.forward(x_f32, in_scale)
        y = torch.empty(self.nv[0], device=self.dev, dtype=torch.float32)
        gpair_unpack_output(out, self.nv[0], COUT_PAD, out_scale, relu, y)
        return y

    def state_dict(self):
        return {"w": {k: v.cpu() for k, v in self.w32.items()}, "b": {k: v.cpu() for k, v in self.b32.items()},
                "t": self.t}

    def load_state_dict(self, sd):
        for k in self.w32:
            self.w32[k].copy_(sd["w"][k])
            self.wbf[k].copy_(self.w32[k].to(torch.bfloat16))
            self.b32[k].copy_(sd["b"][k])
        self.t = sd["t"]


def conv_bench(dims, cin, cout, modes=(1, 2, 0), reps=20, seed=0, which="fwd"):
    """Time one convolution pass (3 x 3 x 3 taps) on random BF16 data for each convolution path
    mode (see gpair_unet_tensor_path): which = "fwd" (with ReLU), "dgrad" or "wgrad" (weight
    gradient only).  Returns {mode: (ms, TFLOP/s)}."""
    D, H, W = dims
    n = D * H * W
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(n, cin, device="cuda", generator=g).to(torch.bfloat16)
    w = (0.1 * torch.randn(cout, 27, cin, device="cuda", generator=g)).to(torch.bfloat16)
    y = torch.empty(n, cout, device="cuda", dtype=torch.bfloat16)
    gy = torch.randn(n, cout, device="cuda", generator=g).to(torch.bfloat16)
    gx = torch.empty(n, cin, device="cuda", dtype=torch.bfloat16)
    wt = torch.empty(cout * 27 * cin, device="cuda", dtype=torch.bfloat16)
    dw = torch.zeros(cout, 27, cin, device="cuda")
    run = {"fwd": lambda: gpair_conv3d_fwd(x, dims, cin, w, None, cout, 27, True, y),
           "dgrad": lambda: gpair_conv3d_dgrad(gy, dims, cout, w, cin, 27, wt, gx),
           "wgrad": lambda: gpair_conv3d_wgrad(x, gy, dims, cin, cout, 27, dw, None)}[which]
    prev = gpair_unet_tensor_path(-1)
    out = {}
    try:
        for mode in modes:
            gpair_unet_tensor_path(mode)
            run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                run()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[mode] = (ms, 2.0 * n * cout * 27 * cin / (ms * 1e-3) / 1e12)
    finally:
        gpair_unet_tensor_path(prev)
    return out


def train_bench(dims, reps=20, seed=0):
    """Time the network's training step (forward, backward, Adam) and its prediction on random
    input and target volumes, after three warm-up steps.  Returns (train ms, predict ms)."""
    net = UNet3D(dims, seed=seed)
    n = dims[0] * dims[1] * dims[2]
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.rand(n, device="cuda", generator=g)
    t = torch.rand(n, device="cuda", generator=g)
    for _ in range(3):
        net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    for _ in range(reps):
        net.train_step(x, t, 1e-4)
    e1.record()
    for _ in range(reps):
        net.predict(x)
    e2.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, e1.elapsed_time(e2) / reps


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="time one U-Net convolution layer on each kernel path, or the "
                                             "whole training step")
    g = ap.add_mutually_exclusive_group(required=True)
    g.add_argument("--conv-bench", nargs=5, type=int, metavar=("D", "H", "W", "CIN", "COUT"))
    g.add_argument("--train-bench", nargs=3, type=int, metavar=("D", "H", "W"))
    ap.add_argument("--modes", type=int, nargs="+", default=[1, 2, 0])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--pass", dest="which", choices=["fwd", "dgrad", "wgrad"], default="fwd")
    a = ap.parse_args()
    if a.train_bench:
        tr, pr = train_bench(tuple(a.train_bench), a.reps)
        print(json.dumps({"train_step_ms": tr, "predict_ms": pr}))
    else:
        D, H, W, cin, cout = a.conv_bench
        res = conv_bench((D, H, W), cin, cout, tuple(a.modes), a.reps, which=a.which)
        print(json.dumps({f"mode{m}": {"ms": v[0], "TFLOP/s": v[1]} for m, v in res.items()}))
