"""torch.autograd interface to the CUDA step.

`Renderer.render(scenes)` returns the rendered views as a differentiable
tensor (pixels x 3, views concatenated).  Its backward runs the library's
own rasterization backward and projection backward (gs_raster_bwd, then
gs_project_bwd_adam in gradient-only mode); nothing is differentiated by
torch.  Transmittance is recomputed in the backward from the per-pixel final
transmittance, not stored per pair.

The differentiable inputs are the stored parameter tensors of each scene:
geom (3, n, 4) float32 -- mean, quaternion, activated scales and opacity --
and sh (12, n, 4) float32 or (6, n, 8) bfloat16.  Gradients come back in the
same layout and dtype, with respect to the stored (activated) values.
"""
from __future__ import annotations

import torch

from . import gsstep
from .step import camera_params


class Renderer:
    def __init__(self, scene_sizes, cameras, capacity: int = 0, tile=(16, 16), bwd_impl: int = 0,
                 bwd_batch: int = 0, sh_bf16: bool = False, bg=None, device="cuda", threads_per_tile: int = 0):
        self.device = torch.device(device)
        flags = gsstep.STORE_SH_BF16 if sh_bf16 else 0
        self.plan = gsstep.Plan(list(scene_sizes), [(c.width, c.height, c.scene) for c in cameras], capacity,
                                tile, bwd_batch, flags, bwd_impl, threads_per_tile)
        self.ws = torch.empty(self.plan.workspace_bytes(), dtype=torch.uint8, device=self.device)
        gsstep.gs_workspace_init(self.plan, self.ws)
        self.cams = torch.from_numpy(camera_params(cameras)).to(self.device)
        self.bg = None if bg is None else torch.tensor(bg, dtype=torch.float32, device=self.device)
        self.scene_sizes = [int(n) for n in scene_sizes]
        self.view_shapes = [(c.width, c.height) for c in cameras]
        self.sh_bf16 = sh_bf16
        self.generation = 0   # forward calls so far; the workspace holds the last one

    def set_cameras(self, cameras):
        self.cams.copy_(torch.from_numpy(camera_params(cameras)))

    def render(self, scenes):
        """scenes: list of (geom, sh) tensors, one pair per scene."""
        flat = []
        for g, s in scenes:
            flat += [g, s]
        return _GSRender.apply(self, *flat)

    def views(self, image):
        out, o = [], 0
        for (w, h) in self.view_shapes:
            out.append(image[o:o + w * h].view(h, w, 3))
            o += w * h
        return out


class _Bufs:
    """Duck-typed scene buffers for the binding (no moments: gradient mode)."""

    def __init__(self, n, geom, sh):
        self.n, self.geom, self.sh, self.m, self.v = n, geom, sh, None, None


class _GSRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer: Renderer, *flat):
        bufs = []
        for i, n in enumerate(renderer.scene_sizes):
            geom, sh = flat[2 * i].contiguous(), flat[2 * i + 1].contiguous()
            bufs.append(_Bufs(n, geom, sh))
        image = torch.empty((renderer.plan.pixels, 3), dtype=torch.float32, device=renderer.device)
        gsstep.gs_project_fwd(renderer.plan, renderer.ws, bufs, renderer.cams)
        gsstep.gs_bin_sort(renderer.plan, renderer.ws)
        gsstep.gs_raster_fwd(renderer.plan, renderer.ws, renderer.bg, image)
        renderer.generation += 1
        ctx.generation = renderer.generation
        ctx.renderer = renderer
        ctx.bufs = bufs
        ctx.save_for_backward(image)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        r: Renderer = ctx.renderer
        if ctx.generation != r.generation:
            raise RuntimeError("the renderer's workspace holds a later forward; back-propagate each render "
                               "before rendering again with the same Renderer")
        (image,) = ctx.saved_tensors
        dl = grad_image.contiguous().float()
        gsstep.gs_raster_bwd(r.plan, r.ws, image, dl)
        N = sum(r.scene_sizes)
        go = torch.empty((15, N, 4), dtype=torch.float32, device=r.device)
        gsstep.gs_project_bwd_adam(r.plan, r.ws, ctx.bufs, r.cams, None, go)
        grads = [None]
        base = 0
        for b in ctx.bufs:
            n = b.n
            dgeom = go[0:3, base:base + n].contiguous()
            dsh = go[3:15, base:base + n]
            if b.sh.dtype == torch.bfloat16:
                dsh = dsh.reshape(6, 2, n, 4).permute(0, 2, 1, 3).reshape(6, n, 8).to(torch.bfloat16)
            grads += [dgeom, dsh.contiguous()]
            base += n
        return tuple(grads)
