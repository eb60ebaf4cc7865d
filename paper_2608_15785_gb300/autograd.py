"""torch.autograd.Function over the exact-mode render and its hand-written backward.

Forward: rg_scene_create (FP32 storage) + rg_render in exact mode. Backward:
rg_backward, which replays the front end and each pixel's blend on the GPU and
returns the gradients of the FP32 attributes. Argument marshalling only.
"""
from __future__ import annotations

from types import SimpleNamespace

import torch

from .binding import RG_STORE_FP32, Scene


class RenderExact(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, cam, sh_degree=3):
        sc = SimpleNamespace(means=means.detach(), scales=scales.detach(), quats=quats.detach(),
                             opacities=opacities.detach(), sh=sh.detach(), sh_degree=int(sh_degree))
        scene = Scene(sc, storage=RG_STORE_FP32)
        img = scene.render(cam, mode="exact")
        ctx.scene = scene
        ctx.cam = cam
        return img

    @staticmethod
    def backward(ctx, grad_img):
        g = ctx.scene.backward(ctx.cam, grad_img)
        ctx.scene.close()
        return g["means"], g["scales"], g["quats"], g["opacities"], g["sh"], None, None


def render_exact(means, scales, quats, opacities, sh, cam, sh_degree: int = 3):
    """Differentiable exact-mode render: returns a [3, H, W] image."""
    return RenderExact.apply(means, scales, quats, opacities, sh, cam, sh_degree)
