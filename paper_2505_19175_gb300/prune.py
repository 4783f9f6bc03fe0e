"""Pruning rules of Sec. 3.3 ("Pruning") over the per-(view, triangle) statistics that
the forward render gathers (``Context.render_fwd(..., stats=...)`` /
``tri_render_fwd_stats``): a triangle is kept when

  * its largest blending weight T o over all training views reaches ``tau_prune``, and
  * it was composited at more than one pixel (``min_pixels`` = 2) in at least
    ``min_views`` = 2 views ("rendered at least twice with more than one pixel").

The statistics of several render calls (batches of views) are folded with
``PruneStats.update``; ``keep_mask`` decides from [views, triangles] arrays directly.
Works with numpy arrays and torch tensors alike.
"""
from __future__ import annotations


def _xp(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return torch
    except ImportError:     # pragma: no cover
        pass
    import numpy
    return numpy


def keep_mask(max_weight, n_pix, tau_prune: float, min_views: int = 2, min_pixels: int = 2):
    """Boolean keep mask [N] from per-view statistics max_weight [V, N], n_pix [V, N]."""
    xp = _xp(max_weight)
    if xp.__name__ == "torch":
        best = max_weight.max(dim=0).values
        views = (n_pix >= min_pixels).sum(dim=0)
    else:
        best = max_weight.max(axis=0)
        views = (n_pix >= min_pixels).sum(axis=0)
    return (best >= tau_prune) & (views >= min_views)


class PruneStats:
    """Running statistics of one scene over training views: the largest weight seen and
    the number of views in which each triangle covered at least ``min_pixels`` pixels."""

    def __init__(self, n: int, device=None, min_pixels: int = 2):
        import torch
        self.n = int(n)
        self.min_pixels = int(min_pixels)
        self.max_weight = torch.zeros(self.n, device=device)
        self.views = torch.zeros(self.n, dtype=torch.int32, device=device)

    def update(self, max_weight, n_pix) -> None:
        """Fold the [V * N] (view-major) outputs of one render call."""
        mw = max_weight.reshape(-1, self.n)
        npx = n_pix.reshape(-1, self.n)
        self.max_weight = self.max_weight.maximum(mw.max(dim=0).values)
        self.views += (npx >= self.min_pixels).sum(dim=0).to(self.views.dtype)

    def keep(self, tau_prune: float, min_views: int = 2):
        return (self.max_weight >= tau_prune) & (self.views >= min_views)

    def reset(self) -> None:
        self.max_weight.zero_()
        self.views.zero_()
