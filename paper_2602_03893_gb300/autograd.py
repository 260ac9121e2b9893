"""torch.autograd wrappers of the forward operator (Methods: the operators are used as custom
autograd functions).  Forward calls gpair_forward; backward calls gpair_adjoint with the incoming
signal gradient, which returns dL/dA and, when requested, dL/dc and dL/dsigma.  Only the inputs
are saved: every pair window is recomputed in the backward pass, nothing per pair is stored.
"""
from __future__ import annotations

import torch

from . import _lib


def _f32(t: torch.Tensor) -> torch.Tensor:
    return t.detach().to(dtype=torch.float32).contiguous()


class GaussianSignals(torch.autograd.Function):
    """y = A(A, c, sigma) for free Gaussians (structure-of-arrays layout)."""

    @staticmethod
    def forward(ctx, A, cx, cy, cz, sigma, arr: _lib.SensorArray):
        A_, cx_, cy_, cz_, s_ = (_f32(t) for t in (A, cx, cy, cz, sigma))
        g = _lib.Gaussians(A=A_, cx=cx_, cy=cy_, cz=cz_, sigma=s_)
        y = torch.empty((arr.n_sensors, arr.n_samples), device=A.device, dtype=torch.float32)
        _lib.gpair_forward(g, arr, y)
        ctx.save_for_backward(A_, cx_, cy_, cz_, s_)
        ctx.arr = arr
        return y

    @staticmethod
    def backward(ctx, gy):
        A_, cx_, cy_, cz_, s_ = ctx.saved_tensors
        need_geom = any(ctx.needs_input_grad[1:5])
        g = _lib.Gaussians(A=A_, cx=cx_, cy=cy_, cz=cz_, sigma=s_)
        M = A_.numel()
        gA = torch.empty(M, device=A_.device, dtype=torch.float32)
        gc = torch.empty((3, M), device=A_.device, dtype=torch.float32) if need_geom else None
        gs = torch.empty(M, device=A_.device, dtype=torch.float32) if need_geom else None
        _lib.gpair_adjoint(g, ctx.arr, _f32(gy), gA, gc, gs)
        out_c = (gc[0], gc[1], gc[2]) if need_geom else (None, None, None)
        return (gA if ctx.needs_input_grad[0] else None, *out_c, gs if need_geom else None, None)


class GridSignals(torch.autograd.Function):
    """y = A(A) for Gaussians on a grid with a shared sigma (amplitudes only)."""

    @staticmethod
    def forward(ctx, A, grid: _lib.Grid, arr: _lib.SensorArray):
        A_ = _f32(A)
        y = torch.empty((arr.n_sensors, arr.n_samples), device=A.device, dtype=torch.float32)
        _lib.gpair_forward(_lib.Gaussians(A=A_, grid=grid), arr, y)
        ctx.grid, ctx.arr, ctx.M = grid, arr, A_.numel()
        ctx.save_for_backward(A_)
        return y.view(arr.n_sensors, arr.n_samples)

    @staticmethod
    def backward(ctx, gy):
        (A_,) = ctx.saved_tensors
        gA = torch.empty(ctx.M, device=A_.device, dtype=torch.float32)
        _lib.gpair_adjoint(_lib.Gaussians(A=A_, grid=ctx.grid), ctx.arr, _f32(gy), gA)
        return gA.view_as(A_), None, None


def gaussian_signals(A, cx, cy, cz, sigma, arr):
    return GaussianSignals.apply(A, cx, cy, cz, sigma, arr)


def grid_signals(A, grid, arr):
    return GridSignals.apply(A, grid, arr)
