"""Pruning rule of Sec. 3.3 ("Pruning") on device tensors: thin wrappers of
``tri_prune_fold`` / ``tri_prune_mask`` over the per-(view, triangle) statistics that
the forward render gathers (``Context.render_fwd(..., stats=...)`` /
``tri_render_fwd_stats``). A triangle is kept when

  * its largest blending weight T o over all training views reaches ``tau_prune``, and
  * it was composited at more than one pixel (``min_pixels`` = 2) in at least
    ``min_views`` = 2 views ("rendered at least twice with more than one pixel").

The statistics of several render calls (batches of views) are folded with
``PruneStats.update``; ``keep_mask`` decides from [views, triangles] tensors directly.
Every reduction runs in the library's kernels; this module only passes pointers.
"""
from __future__ import annotations

import torch

from . import native as N


def _check(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == dtype):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


def _fold(max_weight, n_pix, n: int, min_pixels: int, best, views) -> None:
    _check(max_weight, torch.float32, "max_weight")
    _check(n_pix, torch.int32, "n_pix")
    if max_weight.numel() != n_pix.numel() or max_weight.numel() % max(n, 1):
        raise ValueError("max_weight and n_pix must both hold [views, n] entries")
    nviews = max_weight.numel() // max(n, 1)
    stream = torch.cuda.current_stream(best.device).cuda_stream
    N.check(N.lib().tri_prune_fold(max_weight.data_ptr(), n_pix.data_ptr(), int(nviews), int(n), int(min_pixels),
                                   best.data_ptr(), views.data_ptr(), stream))


def _mask(best, views, tau_prune: float, min_views: int):
    keep = torch.empty(best.numel(), dtype=torch.uint8, device=best.device)
    stream = torch.cuda.current_stream(best.device).cuda_stream
    N.check(N.lib().tri_prune_mask(best.data_ptr(), views.data_ptr(), int(best.numel()), float(tau_prune),
                                   int(min_views), keep.data_ptr(), stream))
    return keep.bool()


def keep_mask(max_weight, n_pix, tau_prune: float, min_views: int = 2, min_pixels: int = 2):
    """Boolean keep mask [N] (device) from per-view statistics max_weight [V, N] and
    n_pix [V, N] (device float32 / int32)."""
    n = int(max_weight.shape[-1])
    best = torch.zeros(n, device=max_weight.device)
    views = torch.zeros(n, dtype=torch.int32, device=max_weight.device)
    _fold(max_weight.contiguous(), n_pix.contiguous(), n, min_pixels, best, views)
    return _mask(best, views, tau_prune, min_views)


class PruneStats:
    """Running statistics of one scene over training views (device): the largest weight
    seen and the number of views in which each triangle covered at least ``min_pixels``
    pixels."""

    def __init__(self, n: int, device=None, min_pixels: int = 2):
        self.n = int(n)
        self.min_pixels = int(min_pixels)
        self.max_weight = torch.zeros(self.n, device=device)
        self.views = torch.zeros(self.n, dtype=torch.int32, device=device)

    def update(self, max_weight, n_pix) -> None:
        """Fold the [V * N] (view-major) outputs of one render call."""
        _fold(max_weight.contiguous(), n_pix.contiguous(), self.n, self.min_pixels, self.max_weight, self.views)

    def keep(self, tau_prune: float, min_views: int = 2):
        return _mask(self.max_weight, self.views, tau_prune, min_views)

    def reset(self) -> None:
        self.max_weight.zero_()
        self.views.zero_()
