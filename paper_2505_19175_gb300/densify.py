"""Densification moves and the size regulariser on device tensors (Sec. 3.3
"Densification", Sec. 3.4 L_s): thin wrappers of ``tri_densify`` / ``tri_size_reg``.
The selection policy (the paper samples by opacity and 1 / sigma) is the caller's."""
from __future__ import annotations

import torch

from . import native as N


def densify(ctx, verts, sh, opacity, sigma, n: int, sel, noise, noise_scale: float, tau_small: float,
            sh_degree: int) -> int:
    """In place on tensors with room for ``n + 3 len(sel)`` triangles (first ``n`` valid):
    subdivide each selected triangle into four, or clone it with in-plane noise when its
    area is below ``tau_small``. Returns the new triangle count (synchronises)."""
    k = int(sel.numel())
    cap = int(verts.shape[0])
    for t in (verts, sh, opacity, sigma, sel, noise):
        if not t.is_contiguous() or not t.is_cuda:
            raise ValueError("densify needs contiguous CUDA tensors")
    if sel.dtype != torch.int32 or noise.dtype != torch.float32 or noise.numel() < 2 * k:
        raise ValueError("sel must be int32 [k], noise float32 [k, 2]")
    n_out = torch.empty(1, dtype=torch.int64, device=verts.device)
    stream = torch.cuda.current_stream().cuda_stream
    N.check(N.lib().tri_densify(ctx.h, verts.data_ptr(), sh.data_ptr(), opacity.data_ptr(), sigma.data_ptr(),
                                int(sh_degree), int(n), cap, sel.data_ptr() if k else None, k,
                                noise.data_ptr() if k else None, float(noise_scale), float(tau_small),
                                n_out.data_ptr(), stream), ctx.h)
    return int(n_out.item())


def size_reg(verts, n: int | None = None, weight: float = 1.0, grad=None):
    """weight * sum 2 / |(v1 - v0) x (v2 - v0)| over the first n triangles (device scalar);
    adds its gradient to ``grad`` when given."""
    n = int(verts.shape[0]) if n is None else int(n)
    loss = torch.empty((), device=verts.device)
    stream = torch.cuda.current_stream().cuda_stream
    N.check(N.lib().tri_size_reg(verts.data_ptr(), n, float(weight), loss.data_ptr(),
                                 grad.data_ptr() if grad is not None else None, stream))
    return loss
