"""Differentiable rendering: a torch.autograd.Function whose backward recomputes the march.

The forward keeps only the per-ray colours it returns; the backward calls dot_render_backward,
which marches every ray again (no per-sample state is stored) and scatters FP32 gradients into
the leaves.  Leaf parameters live in the tree in their storage type (FP32 / FP16 / BF16), so the
gradients are delivered to FP32 "gradient sinks": zero tensors shaped like sigma [L] and
sh [L, 3, K] that take part in the graph only to receive dL/dsigma and dL/dsh.
"""
from __future__ import annotations

import torch

from . import dot


class DotRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_sink, sh_sink, tree, rays, opts):
        R = dot.n_rays_of(rays)
        rgb = torch.empty(R, 3, dtype=torch.float32, device="cuda")
        dot.dot_render_forward(tree, rays, opts, rgb)
        ctx.tree, ctx.rays, ctx.opts = tree, rays, opts
        ctx.save_for_backward(rgb)
        return rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        (rgb,) = ctx.saved_tensors
        inf = ctx.tree.info()
        gs = torch.zeros(inf.n_leaves, dtype=torch.float32, device="cuda")
        gsh = torch.zeros(inf.n_leaves, 3, inf.n_coeffs, dtype=torch.float32, device="cuda")
        dot.dot_render_backward(ctx.tree, ctx.rays, ctx.opts, grad_rgb.contiguous(), rgb, gs, gsh)
        return gs, gsh, None, None, None


def gradient_sinks(tree: dot.Octree):
    """FP32 zero tensors (requires_grad) that receive dL/dsigma [L] and dL/dsh [L, 3, K]."""
    inf = tree.info()
    s = torch.zeros(inf.n_leaves, dtype=torch.float32, device="cuda", requires_grad=True)
    h = torch.zeros(inf.n_leaves, 3, inf.n_coeffs, dtype=torch.float32, device="cuda",
                    requires_grad=True)
    return s, h


def render(tree: dot.Octree, rays, opts, sinks=None) -> torch.Tensor:
    """Differentiable render of `rays`: returns rgb [R, 3]; gradients land in `sinks`."""
    if sinks is None:
        sinks = gradient_sinks(tree)
    return DotRender.apply(sinks[0], sinks[1], tree, rays, opts)
