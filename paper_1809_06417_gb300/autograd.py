"""torch.autograd.Function over the rendering entry points.

Forward: fr_render (Eqs. 5-8, with temperature records mapped to RGB through
the colour-temperature table of Sec. 3.3.3).  Backward: fr_render_backward,
the exact gradient of the rendered images with transmittance recomputed along
each ray from the rendered radiance (nothing per sample is stored).
"""
from __future__ import annotations

import torch

from . import flamerec as fr


class FlameRender(torch.autograd.Function):
    """images = FlameRender.apply(vol, scene)

    vol: (nz, ny, nx, C) CUDA tensor, C = 4 {S_r, S_g, S_b, sigma} for
    kind FR_KIND_RGB or C = 2 {T, sigma} for FR_KIND_TEMP.  scene: a
    RenderScene (cameras, geometry, parameters and the library context).
    Returns (K, H, W, 3) float32 images; the gradient flows to vol."""

    @staticmethod
    def forward(ctx, vol, scene):
        vol = vol.contiguous()
        out = torch.empty(scene.image_shape, device=vol.device, dtype=torch.float32)
        scene.ctx.fr_render(scene.volume(vol), scene.fcams, scene.params, out)
        ctx.scene = scene
        ctx.save_for_backward(vol, out)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        vol, out = ctx.saved_tensors
        scene = ctx.scene
        grad = torch.zeros(vol.shape, device=vol.device, dtype=torch.float32)
        scene.ctx.fr_render_backward(scene.volume(vol), scene.fcams, scene.params, out,
                                     grad_out.contiguous().float(), grad)
        return grad.to(vol.dtype), None


class RenderScene:
    """Cameras, grid geometry and method parameters for FlameRender."""

    def __init__(self, ctx, cams, origin, h, kind=fr.FR_KIND_RGB, **params):
        self.ctx = ctx
        self.cams = list(cams)
        self.fcams = fr.cameras(self.cams)
        self.origin, self.h, self.kind = origin, h, kind
        self.params = fr.params(**params)
        self._keep = params.get("lut")  # the table must outlive the launches
        W, H = self.cams[0]["width"], self.cams[0]["height"]
        self.image_shape = (len(self.cams), H, W, 3)

    def volume(self, t):
        return fr.volume(t, self.origin, self.h, kind=self.kind)


def render(vol, scene):
    return FlameRender.apply(vol, scene)
