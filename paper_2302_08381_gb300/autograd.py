"""torch.autograd wrappers: forward values through the CUDA library; the
backward is the fused recompute-backward kernel (no [n, 3, K] tensor); its own
backward (for force training) is the double-backward kernel."""

from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import api


class _Backward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, g, l_max, normalized):
        ctx.save_for_backward(xyz, g)
        ctx.l_max = l_max
        ctx.normalized = normalized
        return api.backward(xyz, g, l_max, normalized)

    @staticmethod
    @once_differentiable
    def backward(ctx, v):
        xyz, g = ctx.saved_tensors
        need_xyz, need_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_xyz or need_g):
            return None, None, None, None
        grad_g, grad_xyz = api.double_backward(
            xyz, g, v.contiguous(), ctx.l_max, ctx.normalized, need_g=need_g, need_xyz=need_xyz
        )
        return grad_xyz, grad_g, None, None


class SphericalHarmonicsFn(torch.autograd.Function):
    """sph = Y(xyz) with dL/dxyz from the fused backward kernel."""

    @staticmethod
    def forward(ctx, xyz, l_max, normalized):
        ctx.save_for_backward(xyz)
        ctx.l_max = l_max
        ctx.normalized = normalized
        return api.spherical_harmonics(xyz, l_max, normalized)

    @staticmethod
    def backward(ctx, g):
        (xyz,) = ctx.saved_tensors
        if not ctx.needs_input_grad[0]:
            return None, None, None
        return _Backward.apply(xyz, g.contiguous(), ctx.l_max, ctx.normalized), None, None


def spherical_harmonics_autograd(xyz: torch.Tensor, l_max: int, normalized: bool = False) -> torch.Tensor:
    """Differentiable (twice) spherical harmonics of xyz [n, 3]."""
    return SphericalHarmonicsFn.apply(xyz.contiguous(), l_max, normalized)
