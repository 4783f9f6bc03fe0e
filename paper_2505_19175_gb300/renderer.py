"""Python front end of the native renderer: scenes as CUDA tensors, a context wrapper
over the five pipeline calls, and one-call render / render-with-gradients helpers.

Every step runs in the native library; this module only moves pointers and streams.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import native as N


@dataclass
class SceneTensors:
    """Device-resident scene (fp32, contiguous)."""
    verts: torch.Tensor      # [N, 3, 3]
    sh: torch.Tensor         # [N, (deg+1)^2, 3]
    opacity: torch.Tensor    # [N]
    sigma: torch.Tensor      # [N]
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.verts.shape[0])

    @staticmethod
    def from_numpy(scene, device="cuda") -> "SceneTensors":
        def t(x):
            return torch.as_tensor(np.ascontiguousarray(x, np.float32)).to(device)
        return SceneTensors(t(scene.verts), t(scene.sh), t(scene.opacity), t(scene.sigma), int(scene.sh_degree))

    def check(self) -> None:
        n = self.n
        k = (self.sh_degree + 1) ** 2
        for name, x, shape in (("verts", self.verts, (n, 3, 3)), ("sh", self.sh, (n, k, 3)),
                               ("opacity", self.opacity, (n,)), ("sigma", self.sigma, (n,))):
            if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or tuple(x.shape) != shape:
                raise ValueError(f"{name}: want contiguous float32 CUDA tensor of shape {shape}")

    def as_abi(self) -> N.tri_scene:
        self.check()
        s = N.tri_scene()
        s.verts, s.sh = self.verts.data_ptr(), self.sh.data_ptr()
        s.opacity, s.sigma = self.opacity.data_ptr(), self.sigma.data_ptr()
        s.n, s.sh_degree = self.n, self.sh_degree
        return s


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Context:
    """One tri_ctx: owns the device workspace of one pipeline run at a time."""

    def __init__(self, device: int | None = None):
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._lib = N.lib()
        h = C.c_void_p()
        N.check(self._lib.tri_ctx_create(C.byref(h), self.device))
        self.h = h
        self.cams = None
        self._scene = None        # keeps the scene tensors alive until the backward

    def close(self) -> None:
        if self.h:
            self._lib.tri_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        N.check(st, self.h)

    def reserve(self, pairs: int) -> None:
        self._ck(self._lib.tri_reserve(self.h, int(pairs)))

    def preprocess(self, scene: SceneTensors, cams, stream=None) -> None:
        self.cams = list(cams)
        self._scene = scene
        self._abi_scene = scene.as_abi()
        self._abi_cams = N.camera_array(self.cams)
        self._ck(self._lib.tri_preprocess(self.h, C.byref(self._abi_scene), self._abi_cams, len(self.cams),
                                          _stream_handle(stream)))

    def bin_sort(self, sync: bool = False, stream=None):
        if sync:
            n = C.c_int64()
            self._ck(self._lib.tri_bin_sort(self.h, C.byref(n), _stream_handle(stream)))
            return int(n.value)
        self._ck(self._lib.tri_bin_sort(self.h, None, _stream_handle(stream)))
        return None

    def render_fwd(self, images, T_final=None, n_contrib=None, stream=None, stats=None) -> None:
        """Composite the views into ``images``. With ``stats = (max_weight, n_pixels)``
        (device float32 / int32 tensors of views x triangles entries, view-major) also
        gather the pruning statistics of Sec. 3.3 (see ``prune``)."""
        ims = N.ptr_array([x.data_ptr() for x in images])
        tf = N.ptr_array([x.data_ptr() for x in T_final]) if T_final is not None else None
        nc = N.ptr_array([x.data_ptr() for x in n_contrib]) if n_contrib is not None else None
        if stats is None:
            self._ck(self._lib.tri_render_fwd(self.h, ims, tf, nc, _stream_handle(stream)))
        else:
            mw, npx = stats
            n_items = len(self.cams) * self._scene.n
            if mw.numel() < n_items or npx.numel() < n_items or mw.dtype != torch.float32 or npx.dtype != torch.int32:
                raise ValueError("stats need float32 and int32 tensors of views x triangles entries")
            self._ck(self._lib.tri_render_fwd_stats(self.h, ims, tf, nc, mw.data_ptr(), npx.data_ptr(),
                                                    _stream_handle(stream)))

    def render_fwd_l1(self, images, targets, grads, loss=None, stream=None) -> None:
        """Composite the views into ``images`` and, in the same kernel, write the L1
        loss gradient sign(image - target) / n into ``grads`` and (if given) the mean
        absolute difference into the device scalar ``loss`` (n = all views' values)."""
        ims = N.ptr_array([x.data_ptr() for x in images])
        tg = N.ptr_array([x.data_ptr() for x in targets])
        gr = N.ptr_array([x.data_ptr() for x in grads])
        self._ck(self._lib.tri_render_fwd_l1(self.h, ims, tg, gr, loss.data_ptr() if loss is not None else None,
                                             _stream_handle(stream)))

    def set_window(self, window: int) -> None:
        """Window of the next preprocess: ``native.WINDOW_POWER`` (Eq. indicator1, the
        default) or ``native.WINDOW_SIGMOID`` (Eq. indicator2)."""
        self._ck(self._lib.tri_set_window(self.h, int(window)))

    def set_fragment_counting(self, on: bool) -> None:
        """Count the forward's evaluated and composited fragments into ``info()``
        (off by default)."""
        self._ck(self._lib.tri_set_fragment_counting(self.h, int(bool(on))))

    def set_sort(self, sort: int) -> None:
        """Compositing order of the next preprocess: ``native.SORT_TILE`` (per tile by
        centroid depth, the default) or ``native.SORT_PIXEL`` (per pixel by the depth of
        the triangle's plane along the pixel's ray)."""
        self._ck(self._lib.tri_set_sort(self.h, int(sort)))

    def render_solid(self, scene: SceneTensors, cams, images, ids=None, sync_pairs: bool = True,
                     stream=None) -> int:
        """Opaque-triangle render of ``cams`` into ``images`` (and the winning triangle
        index per pixel into ``ids``, int32 [H,W] tensors, -1 for background). Returns
        the pair count when ``sync_pairs`` (growing the pair list if needed), else -1."""
        self.cams = list(cams)
        self._scene = scene
        self._abi_scene = scene.as_abi()
        self._abi_cams = N.camera_array(self.cams)
        ims = N.ptr_array([x.data_ptr() for x in images])
        idp = N.ptr_array([x.data_ptr() for x in ids]) if ids is not None else None
        n = C.c_int64(-1)
        self._ck(self._lib.tri_render_solid(self.h, C.byref(self._abi_scene), self._abi_cams, len(self.cams), ims,
                                            idp, C.byref(n) if sync_pairs else None, _stream_handle(stream)))
        return int(n.value)

    def render_bwd(self, dL_dimages, stream=None) -> None:
        self._dl = [x.contiguous() for x in dL_dimages]
        self._ck(self._lib.tri_render_bwd(self.h, N.ptr_array([x.data_ptr() for x in self._dl]),
                                          _stream_handle(stream)))

    def preprocess_bwd(self, dverts=None, dsh=None, dopacity=None, dsigma=None, accumulate=False,
                       stream=None) -> None:
        p = lambda x: None if x is None else x.data_ptr()  # noqa: E731
        self._ck(self._lib.tri_preprocess_bwd(self.h, p(dverts), p(dsh), p(dopacity), p(dsigma),
                                              int(bool(accumulate)), _stream_handle(stream)))

    def check(self, stream=None) -> N.tri_ctx_info:
        info = N.tri_ctx_info()
        self._ck(self._lib.tri_ctx_check(self.h, C.byref(info), _stream_handle(stream)))
        return info

    def info(self, stream=None) -> N.tri_ctx_info:
        """Counters without raising on an overflow or device-side error."""
        info = N.tri_ctx_info()
        self._lib.tri_ctx_check(self.h, C.byref(info), _stream_handle(stream))
        return info

    _DEBUG = {"pair_tiles": (0, np.uint32, 1), "pair_items": (1, np.uint32, 1), "ranges": (2, np.uint32, 2),
              "depth_keys": (3, np.uint32, 1), "rects": (4, np.uint16, 4), "ntiles": (5, np.uint32, 1),
              "binned": (6, np.uint64, 1), "records": (7, np.float32, 16), "grad2d": (8, np.float32, 16),
              "tile_order": (9, np.uint32, 1)}

    def debug_withhold_scan(self, cta: int = 0, wait_ns: int = 0) -> None:
        """Failure-detection test hook: the next bin_sort's scan leaves the look-back
        word of CTA ``cta`` unset and its bounded waits give up after ``wait_ns``."""
        self._ck(self._lib.tri_debug_withhold_scan(self.h, int(cta), int(wait_ns)))

    def debug(self, name: str) -> np.ndarray:
        which, dt, width = self._DEBUG[name]
        info = self.info()
        cap = max(info.n_items, info.n_pairs, info.total_tiles, 1) * 64 + 64
        buf = np.empty(cap, np.uint8)
        used = C.c_size_t()
        self._ck(self._lib.tri_debug_copy(self.h, which, buf.ctypes.data_as(C.c_void_p), buf.nbytes,
                                          C.byref(used)))
        out = buf[:used.value].view(dt)
        return out.reshape(-1, width) if width > 1 else out


def new_images(cams, device="cuda"):
    return [torch.empty((3, int(N._get(c, "H")), int(N._get(c, "W"))), device=device, dtype=torch.float32)
            for c in cams]


def render(scene: SceneTensors, cams, ctx: Context | None = None, sync_pairs: bool = True, stream=None):
    """Images [3,H,W] of each camera (forward only)."""
    ctx = ctx or Context()
    ctx.preprocess(scene, cams, stream)
    ctx.bin_sort(sync=sync_pairs, stream=stream)
    imgs = new_images(cams, scene.verts.device)
    ctx.render_fwd(imgs, stream=stream)
    return imgs


def loss_l1(image: torch.Tensor, target: torch.Tensor, stream=None):
    """(mean |image - target| as a device scalar, dL/dimage) from the native kernel."""
    grad = torch.empty_like(image)
    loss = torch.empty((), device=image.device, dtype=torch.float32)
    N.check(N.lib().tri_loss_l1(image.data_ptr(), target.contiguous().data_ptr(), image.numel(),
                                grad.data_ptr(), loss.data_ptr(), _stream_handle(stream)))
    return loss, grad
