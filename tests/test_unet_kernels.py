"""BF16 tensor-core convolution kernels and the U-Net built on them, against FP64 CPU references
(torch.nn.functional.conv3d and autograd in float64 on the same bf16-rounded inputs)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet_ref
from paper_2602_03893_gb300 import unet

pytestmark = pytest.mark.gpu


def _bf(shape, gen, scale=1.0):
    return (torch.randn(shape, generator=gen) * scale).to(torch.bfloat16)


def _cl_to_cf(x_cl, dims):
    D, H, W = dims
    return x_cl.double().reshape(D, H, W, -1).permute(3, 0, 1, 2).unsqueeze(0)


def _cf_to_cl(x_cf):
    return x_cf.squeeze(0).permute(1, 2, 3, 0).reshape(-1, x_cf.shape[1])


def _close(got, ref, rel=2e-2):
    got = got.double().cpu()
    ref = ref.double().cpu()
    err = (got - ref).norm() / max(ref.norm().item(), 1e-30)
    assert err < rel, f"rel err {err:.3e}"
    return err


@pytest.mark.parametrize("dims,cin,cout,taps,relu", [((6, 5, 7), 16, 16, 27, True), ((4, 6, 5), 48, 32, 27, False),
                                                      ((5, 4, 9), 32, 128, 27, True), ((3, 3, 3), 16, 16, 27, False),
                                                      ((7, 5, 6), 64, 48, 27, True), ((4, 4, 4), 16, 16, 1, False),
                                                      ((6, 6, 6), 192, 64, 27, True), ((9, 8, 7), 32, 256, 27, True)])
@pytest.mark.parametrize("path", [2, 0])
def test_conv_fwd_dgrad_wgrad(dims, cin, cout, taps, relu, path):
    """path 2: the tcgen05 kernel (every shape here is eligible), path 0: the mma.sync kernel."""
    prev = unet.gpair_unet_tensor_path(path)
    try:
        _conv_case(dims, cin, cout, taps, relu)
        assert unet.gpair_unet_tc_status() == 0
    finally:
        unet.gpair_unet_tensor_path(prev)


def _conv_case(dims, cin, cout, taps, relu):
    gen = torch.Generator().manual_seed(cin * 7 + cout)
    nv = int(np.prod(dims))
    x = _bf((nv, cin), gen)
    w = _bf((cout, taps, cin), gen, scale=0.2)
    b = torch.randn(cout, generator=gen).float()
    dout = _bf((nv, cout), gen)
    dev = "cuda"
    xd, wd, bd, gd = x.to(dev), w.to(dev), b.to(dev), dout.to(dev)
    y = torch.empty((nv, cout), dtype=torch.bfloat16, device=dev)
    unet.gpair_conv3d_fwd(xd, dims, cin, wd, bd, cout, taps, relu, y)
    # FP64 reference on the same bf16 values
    xr = _cl_to_cf(x, dims).requires_grad_(True)
    wr = w.double().requires_grad_(True)
    yr = unet_ref.conv(xr, wr, b.double(), taps, relu)
    _close(y.float().cpu(), _cf_to_cl(yr.detach()), rel=1e-2)
    # data and weight gradients of the convolution (before the activation)
    yr_lin = unet_ref.conv(xr, wr, b.double(), taps, False)
    yr_lin.backward(_cl_to_cf(dout, dims))
    din = torch.empty((nv, cin), dtype=torch.bfloat16, device=dev)
    wt = torch.empty(cout * taps * cin, dtype=torch.bfloat16, device=dev)
    unet.gpair_conv3d_dgrad(gd, dims, cout, wd, cin, taps, wt, din)
    _close(din.float().cpu(), _cf_to_cl(xr.grad), rel=1e-2)
    dw = torch.zeros((cout, taps, cin), device=dev)
    db = torch.zeros(cout, device=dev)
    unet.gpair_conv3d_wgrad(xd, gd, dims, cin, cout, taps, dw, db)
    _close(dw.cpu(), wr.grad, rel=1e-4)
    _close(db.cpu(), dout.double().sum(0), rel=1e-4)


def test_tensor_core_paths_agree_on_the_unet_layers():
    """The tcgen05 and mma.sync convolutions on the U-Net's own layer shapes (128 x 128 x 64 level
    halved to keep the test short): both accumulate in FP32, so their BF16 outputs differ by at most
    a few units in the last place."""
    gen = torch.Generator().manual_seed(11)
    dims = (16, 32, 32)
    nv = int(np.prod(dims))
    for cin, cout in [(16, 16), (32, 32), (64, 64), (128, 128), (256, 128), (32, 16)]:
        x = _bf((nv, cin), gen).cuda()
        w = _bf((cout, 27, cin), gen, scale=0.1).cuda()
        b = torch.randn(cout, generator=gen).float().cuda()
        outs = []
        for path in (2, 0):
            prev = unet.gpair_unet_tensor_path(path)
            y = torch.empty((nv, cout), dtype=torch.bfloat16, device="cuda")
            unet.gpair_conv3d_fwd(x, dims, cin, w, b, cout, 27, True, y)
            torch.cuda.synchronize()
            unet.gpair_unet_tensor_path(prev)
            outs.append(y.float())
        assert unet.gpair_unet_tc_status() == 0
        d = (outs[0] - outs[1]).abs()
        scale = outs[1].abs().max().item()
        assert d.max().item() <= 2e-2 * scale, (cin, cout, d.max().item(), scale)
        assert (d > 0).float().mean().item() < 0.2, (cin, cout)


def test_pool_up_concat_relu():
    gen = torch.Generator().manual_seed(3)
    dims, C = (4, 6, 8), 16
    nv = 4 * 6 * 8
    x = _bf((nv, C), gen)
    dev = "cuda"
    xd = x.to(dev)
    p = torch.empty((nv // 8, C), dtype=torch.bfloat16, device=dev)
    unet.gpair_pool2_fwd(xd, dims, C, p)
    ref = _cf_to_cl(F.avg_pool3d(_cl_to_cf(x, dims), 2))
    _close(p.float().cpu(), ref, rel=1e-2)
    u = torch.empty((nv, C), dtype=torch.bfloat16, device=dev)
    unet.gpair_up2_fwd(p, (2, 3, 4), C, u)
    refu = _cf_to_cl(F.interpolate(_cl_to_cf(p.float().cpu(), (2, 3, 4)), scale_factor=2, mode="nearest"))
    _close(u.float().cpu(), refu, rel=1e-6)
    # adjointness of pool / up against their backward kernels: <P x, y> = <x, P^T y>
    yv = _bf((nv // 8, C), gen).to(dev)
    pt = torch.empty((nv, C), dtype=torch.bfloat16, device=dev)
    unet.gpair_pool2_bwd(yv, dims, C, pt)
    lhs = (p.double() * yv.double()).sum()
    rhs = (xd.double() * pt.double()).sum()
    assert abs(lhs - rhs) <= 2e-2 * abs(lhs) + 1e-2
    ub = torch.empty((nv // 8, C), dtype=torch.bfloat16, device=dev)
    unet.gpair_up2_bwd(xd, (2, 3, 4), C, ub)
    lhs2 = (u.double() * xd.double()).sum()
    rhs2 = (p.double() * ub.double()).sum()
    assert abs(lhs2 - rhs2) <= 2e-2 * abs(lhs2) + 1e-2
    a2 = _bf((nv, 8), gen).to(dev)
    cat = torch.empty((nv, C + 8), dtype=torch.bfloat16, device=dev)
    unet.gpair_concat_fwd(xd, C, a2, 8, nv, cat)
    assert torch.equal(cat.cpu(), torch.cat([x, a2.cpu()], 1))
    da = torch.empty_like(xd)
    dbb = torch.empty_like(a2)
    unet.gpair_concat_bwd(cat, C, 8, nv, da, dbb)
    assert torch.equal(da, xd) and torch.equal(dbb, a2)
    g = torch.ones_like(xd)
    unet.gpair_relu_bwd(xd, g)
    assert torch.equal(g.cpu(), (x.float() > 0).to(torch.bfloat16))


def test_unet_forward_backward_matches_fp64_reference():
    """The whole network against the FP64 reference that stores activations and gradients in BF16
    as the kernels do.  Layer by layer (each convolution's weight and data gradient recomputed in
    FP64 from the kernels' own stored BF16 input and masked output gradient) the kernels agree to
    FP32 accumulation (weight gradients, 1e-5) and to the BF16 rounding of their output (data
    gradients, 3e-3).  Through the whole 15-layer network those independent BF16 roundings
    compound: the output agrees to 1e-2 and every layer's weight and bias gradient to 8e-2 (measured:
    3e-3 on the output; 2e-4 to 5.3e-2 on the weight gradients, largest at the bottleneck)."""
    dims = (8, 16, 16)
    net = unet.UNet3D(dims, seed=1)
    gen = torch.Generator().manual_seed(5)
    nv = int(np.prod(dims))
    x = torch.randn(nv, generator=gen).float()
    target = torch.rand(nv, generator=gen).float()
    out = net.forward(x.cuda(), 1.0).float().cpu()
    W = {k: v.cpu().to(torch.bfloat16).double().requires_grad_(True) for k, v in net.w32.items()}
    B = {k: v.cpu().double().requires_grad_(True) for k, v in net.b32.items()}
    x0 = torch.zeros((1, unet.CIN_PAD) + dims, dtype=torch.float64)
    x0[0, 0] = x.to(torch.bfloat16).double().reshape(dims)
    ref = unet_ref.unet_forward(x0, W, B, bf16_storage=True)
    _close(out[:, 0], ref[0, 0].reshape(-1).detach(), rel=1e-2)
    # gradients of the same MSE loss on channel 0
    loss = torch.mean((ref[0, 0].reshape(-1) - target.double()) ** 2)
    loss.backward()
    net.loss.zero_()
    unet.gpair_mse_loss(net.act["out"], target.cuda(), nv, unet.COUT_PAD, net.grad["out"], net.loss)
    net.backward(net.grad["out"])
    assert abs(net.loss.item() / nv - loss.item()) <= 1e-2 * loss.item()
    for name in unet_ref.ORDER:
        _close(net.gw[name].cpu(), W[name].grad, rel=8e-2)
        _close(net.gb[name].cpu(), B[name].grad, rel=8e-2)
    # layer by layer on the kernels' own stored tensors (relu_bwd has masked net.grad in place)
    lv = [(dims[0] >> q, dims[1] >> q, dims[2] >> q) for q in range(4)]
    inputs = {"e1a": ("x", 0), "e1b": ("e1a", 0), "e2a": ("p1", 1), "e2b": ("e2a", 1), "e3a": ("p2", 2),
              "e3b": ("e3a", 2), "b4a": ("p3", 3), "b4b": ("b4a", 3), "d3a": ("k3", 2), "d3b": ("d3a", 2),
              "d2a": ("k2", 1), "d2b": ("d2a", 1), "d1a": ("k1", 0), "d1b": ("d1a", 0), "out": ("d1b", 0)}
    assert set(inputs) == set(unet_ref.ORDER)
    for name, (src, l) in inputs.items():
        c = net.convs[name]
        xin = _cl_to_cf(net.act[src].cpu(), lv[l]).requires_grad_(True)
        wr = net.wbf[name].cpu().double().requires_grad_(True)
        y = unet_ref.conv(xin, wr, net.b32[name].cpu().double(), c.taps, False)
        y.backward(_cl_to_cf(net.grad[name].cpu(), lv[l]))
        _close(net.gw[name].cpu(), wr.grad, rel=1e-5)
        if name != "e1a":
            gin = xin.grad
            if src in net.convs and net.convs[src].relu:
                gin = gin * (_cl_to_cf(net.act[src].cpu(), lv[l]) > 0)
            _close(_cl_to_cf(net.grad[src].cpu(), lv[l]), gin, rel=3e-3)


def test_training_reduces_loss():
    dims = (8, 16, 16)
    net = unet.UNet3D(dims, seed=2)
    gen = torch.Generator().manual_seed(7)
    nv = int(np.prod(dims))
    xs = [torch.randn(nv, generator=gen).float().cuda() for _ in range(4)]
    ts = [torch.relu(x * 0.5 + 0.2) for x in xs]
    first = last = None
    for it in range(60):
        l = float(net.train_step(xs[it % 4], ts[it % 4], 3e-3).item()) / nv
        first = l if first is None else first
        last = l
    assert last < 0.3 * first, (first, last)
