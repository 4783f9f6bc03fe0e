"""``torch.autograd.Function`` over the native forward / backward passes.

The forward keeps no per-pixel fragment lists: the context holds the sorted tile
lists, each pixel's final transmittance and last composited index, and each tile's
largest index, from which the backward recomputes every alpha and transmittance.
"""
from __future__ import annotations

import threading

import torch

from .renderer import Context, SceneTensors, new_images


class _ContextPool:
    """Contexts are reused across iterations so their workspace stays allocated."""

    def __init__(self):
        self._free = []
        self._lock = threading.Lock()

    def get(self) -> Context:
        with self._lock:
            if self._free:
                return self._free.pop()
        return Context()

    def put(self, ctx: Context) -> None:
        with self._lock:
            self._free.append(ctx)


POOL = _ContextPool()


class TriRasterize(torch.autograd.Function):
    @staticmethod
    def forward(actx, verts, sh, opacity, sigma, sh_degree, cams):
        scene = SceneTensors(verts.detach().contiguous(), sh.detach().contiguous(),
                             opacity.detach().contiguous(), sigma.detach().contiguous(), int(sh_degree))
        rctx = POOL.get()
        rctx.preprocess(scene, cams)
        rctx.bin_sort(sync=True)
        imgs = new_images(cams, verts.device)
        rctx.render_fwd(imgs)
        actx.rctx = rctx
        actx.scene = scene
        return tuple(imgs)

    @staticmethod
    def backward(actx, *grads):
        rctx, scene = actx.rctx, actx.scene
        dls = [g.contiguous() if g is not None else torch.zeros((3, int(c.H), int(c.W)), device=scene.verts.device)
               for g, c in zip(grads, rctx.cams)]
        rctx.render_bwd(dls)
        dv = torch.empty_like(scene.verts)
        dsh = torch.empty_like(scene.sh)
        do = torch.empty_like(scene.opacity)
        ds = torch.empty_like(scene.sigma)
        rctx.preprocess_bwd(dv, dsh, do, ds)
        POOL.put(rctx)
        actx.rctx = None
        return dv, dsh, do, ds, None, None


def rasterize(verts, sh, opacity, sigma, sh_degree, cams):
    """Differentiable render of ``cams`` (a list of cameras); returns one [3,H,W]
    image per camera. Gradients flow to verts, sh, opacity and sigma."""
    return TriRasterize.apply(verts, sh, opacity, sigma, int(sh_degree), tuple(cams))
