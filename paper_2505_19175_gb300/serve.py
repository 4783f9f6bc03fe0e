"""Python front end of the native server (tri_serve_* in include/trisplat.h).

The server keeps scenes resident on the device, admits requests by memory, and batches
camera requests of mixed resolutions into batched launches on several in-flight slots
(continuous batching). This wrapper only marshals arguments and keeps each output
tensor alive until its ticket completes.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np
import torch

from . import native as N


class Server:
    def __init__(self, mem_budget_bytes: int = 0, max_batch: int = 8, max_width: int = 1920,
                 max_height: int = 1080, slots: int = 2, timeout_ms: int = 0, use_graphs: bool = True,
                 batch_window_us: int = 0, graph_after: int = 1, device: int | None = None):
        self._lib = N.lib()
        self.device = torch.cuda.current_device() if device is None else int(device)
        o = N.tri_serve_opts()
        o.mem_budget_bytes = int(mem_budget_bytes)
        o.max_batch, o.max_width, o.max_height = int(max_batch), int(max_width), int(max_height)
        o.slots, o.timeout_ms, o.use_graphs = int(slots), int(timeout_ms), int(bool(use_graphs))
        o.batch_window_us, o.graph_after = int(batch_window_us), int(graph_after)
        h = C.c_void_p()
        N.check(self._lib.tri_serve_create(C.byref(h), C.byref(o), self.device))
        self.h = h
        self._live = {}            # ticket -> output tensor kept alive
        self._lock = threading.Lock()

    def close(self) -> None:
        if self.h:
            self._lib.tri_serve_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scene(self, scene) -> int:
        """Copy a scene (numpy arrays or a SceneTensors) into server memory."""
        s = N.tri_scene()
        if isinstance(scene.verts, torch.Tensor):
            keep = [scene.verts.contiguous(), scene.sh.contiguous(), scene.opacity.contiguous(),
                    scene.sigma.contiguous()]
            ptrs = [x.data_ptr() for x in keep]
        else:
            keep = [np.ascontiguousarray(x, np.float32) for x in (scene.verts, scene.sh, scene.opacity, scene.sigma)]
            ptrs = [x.ctypes.data for x in keep]
        s.verts, s.sh, s.opacity, s.sigma = ptrs
        s.n, s.sh_degree = int(keep[0].shape[0]), int(scene.sh_degree)
        sid = C.c_int32()
        N.check(self._lib.tri_serve_add_scene(self.h, C.byref(s), C.byref(sid)))
        return int(sid.value)

    def remove_scene(self, scene_id: int) -> None:
        N.check(self._lib.tri_serve_remove_scene(self.h, int(scene_id)))

    def submit(self, scene_id: int, cam, out: torch.Tensor | None = None):
        """Queue a render of ``cam``; returns (ticket, output tensor [3,H,W])."""
        if out is None:
            out = torch.empty((3, int(N._get(cam, "H")), int(N._get(cam, "W"))), device=f"cuda:{self.device}")
        t = C.c_uint64()
        N.check(self._lib.tri_serve_submit(self.h, int(scene_id), C.byref(N.make_camera(cam)), out.data_ptr(),
                                           C.byref(t)))
        with self._lock:
            self._live[int(t.value)] = out
        return int(t.value), out

    def poll(self, max_items: int = 4096):
        """[(ticket, status)] of requests finished since the last poll."""
        done = (C.c_uint64 * max_items)()
        st = (C.c_int32 * max_items)()
        n = C.c_int32()
        N.check(self._lib.tri_serve_poll(self.h, done, st, max_items, C.byref(n)))
        out = [(int(done[i]), int(st[i])) for i in range(n.value)]
        with self._lock:
            for t, _ in out:
                self._live.pop(t, None)
        return out

    def wait(self, ticket: int, timeout_ms: int = 60000) -> int:
        """Block until ``ticket`` completes; returns its status (TRI_ERR_TIMEOUT if the wait ran out)."""
        st = int(self._lib.tri_serve_wait(self.h, int(ticket), int(timeout_ms)))
        if st != N.TRI_ERR_TIMEOUT:
            with self._lock:
                self._live.pop(int(ticket), None)
        return st

    def reset_stats(self) -> None:
        N.check(self._lib.tri_serve_reset_stats(self.h))

    def stats(self) -> dict:
        s = N.tri_serve_stats_t()
        N.check(self._lib.tri_serve_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}
