"""Benchmark of the differentiable triangle-splat rasterizer on one GB300.

Default workload (one step = the whole hot path once): 500,000 triangles clustered on
200 planar patches, SH degree 3, one camera at 1297x840, fp32:
    preprocess -> depth sort -> pair emission -> tile sort -> ranges -> render forward
    -> L1 loss against a seeded target -> render backward -> preprocess backward.
The metric is forward+backward iterations per second (device time, CUDA events on the
launching stream, L2 flushed between timed steps); the JSON line also carries the
forward frames per second, the per-stage breakdown, the roofline of the dominant
kernel, an end-to-end number through host buffers, and the FP64 CPU oracle timed on a
bounded sample of the same workload.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) every rank renders its own replica (no collective on the data
path); the value is the sum over ranks of the steps divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd FPS & fwd+bwd it/s at 1297×840, 500k–3M tris; serving p99 ms vs unbatched"
WORKLOAD = "500k tris on 200 planar patches, SH3, 1297x840, 1 view, fwd+bwd with L1 loss"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP32 lanes per SM per clock on the FMA pipe of sm_10x, and MUFU (lg2, ex2, rcp) results
FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16
# The method's work in the render kernels, counted as the method does it (Sec. 3.1):
# every tile-list entry a pixel visits up to its termination (the "contributions per
# pixel", F = sum of n_contrib) costs the three edge-line evaluations, 6 FFMA; only a
# composited fragment (alpha >= 1/255) costs the rest. Forward, per composited
# fragment: sigma lg2, o I, 1 - alpha, alpha T, 3 colour FFMA, the T update -> 7
# FMA-pipe ops and 2 MUFU (lg2, ex2). Backward: the same recomputation + ~30 FMA-pipe
# ops of the adjoint (37) and 1 more MUFU (the reciprocal of 1 - alpha).
ENTRY_OPS = {"fma": 6, "mufu": 0}
COMPOSITED_OPS = {"render_fwd": {"fma": 7, "mufu": 2}, "render_bwd": {"fma": 37, "mufu": 3}}
# The earlier dense count, which charged every entry up to a pixel's last composited one
# with the full per-fragment work; kept beside the real fraction as an effective rate.
DENSE_FRAG_OPS = {"render_fwd": {"fma": 13, "mufu": 2}, "render_bwd": {"fma": 43, "mufu": 3}}


def stage_bytes(n: int, views: int, n_vis: int, pairs: int, pixels: int, sh_floats: int = 48,
                loss: bool = True) -> dict:
    """Algorithmic DRAM bytes of each stage of one step, every buffer read or written once:
    - preprocess: parameters (verts 36 B, SH, o, sigma) read; per triangle its view mask
      (8 B); per visible item its record and rectangle (72 B) and its entry of the
      visible-item list (16 B);
    - bin_sort: per visible item its list entry read (16 B); per pair the binned (key,
      item) word written and read (8 + 8 B) and the sorted item id (4 B);
    - render_fwd: per pair the item id (4 B), the record (64 B) and the group-mask words
      (8 B); per pixel colour, T and count written (20 B), with the L1 loss the target read
      and dL/dimage written (24 B);
    - render_bwd: per pair the item id, the record and one mask word (72 B); per visible
      item its gradient record accumulated (64 B); per pixel T, count and dL/dimage (20 B);
    - preprocess_bwd: parameters read and their gradients written (2 x 236 B at SH
      degree 3); per triangle its view mask (8 B); per visible item its gradient record
      and rounded incenter (80 B)."""
    params = 4 * (9 + sh_floats + 2)
    return {"preprocess": n * params + n * 8 + n_vis * 88,
            "bin_sort": n_vis * 16 + pairs * 20,
            "render_fwd": pairs * 76 + pixels * (44 if loss else 20),
            "render_bwd": pairs * 72 + n_vis * 64 + pixels * 20,
            "preprocess_bwd": 2 * n * params + n * 8 + n_vis * 80}


def stage_gbs(bytes_: dict, ms: dict, hbm_gbs: float) -> dict:
    """Per stage: algorithmic GB/s over the stage's median time and its fraction of the
    measured HBM copy rate."""
    out = {}
    for k, b in bytes_.items():
        t = ms[k] / 1e3
        out[k] = {"bytes": int(b), "gb_s": round(b / t / 1e9, 1), "frac_hbm": round(b / t / 1e9 / hbm_gbs, 4)}
    return out


PROFILE_FILE = os.path.join(ROOT, "profiles", "kernels_patches_500k.md")


def _profiled_traffic(kernel: str):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or None when
    the kernel's source changed after the capture (the sha256 prefix no longer matches)."""
    import hashlib
    try:
        for ln in open(PROFILE_FILE):
            f = ln.split()
            if len(f) == 5 and f[0] == "traffic" and f[1] == kernel:
                with open(os.path.join(ROOT, f[3]), "rb") as src:
                    if hashlib.sha256(src.read()).hexdigest()[:16] == f[4]:
                        return int(f[2])
    except OSError:
        pass
    return None


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region: the
    sampler (100 ms period) is running before the region starts, and the samples kept
    are those taken inside it plus the first one after it (which covers its last
    100 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []          # (time, line)
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            deadline = time.perf_counter() + 5.0
            while not self.lines and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        if self.proc is not None:
            deadline = self.t1 + 0.5
            while time.perf_counter() < deadline and not any(t >= self.t1 for t, _ in self.lines):
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        after = False
        for t, line in list(self.lines):
            if self.t0 is None or t < self.t0:
                continue
            if self.t1 is not None and t >= self.t1:
                if after:
                    break
                after = True
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def make_workload():
    from paper_2505_19175_gb300 import synth
    scene, _, _ = synth.scene_patches()
    cam = synth.camera_patches()
    target = synth.target_image(cam.H, cam.W)
    return scene, cam, target


# ---------------------------------------------------------------------------------------
# CPU oracle: baseline and reference arm
# ---------------------------------------------------------------------------------------
def oracle_sample(scene, cam, target, rows: int):
    """One oracle fwd+bwd over a band of `rows` pixel rows in the image centre (the
    whole frame when rows >= H); returns (seconds, fraction of the frame, threads)."""
    import oracle as O
    mask = None
    if rows < cam.H:
        mask = np.zeros((cam.H, cam.W), np.uint8)
        y0 = cam.H // 2 - rows // 2
        mask[y0:y0 + rows] = 1
    t0 = time.perf_counter()
    ref = O.render(scene, cam, pix_mask=mask)
    g = np.sign(ref["image"] - target) / ref["image"].size
    if mask is not None:
        g = g * mask[None]
    O.render_grad(scene, cam, g, pix_mask=mask)
    dt = time.perf_counter() - t0
    return dt, min(rows, cam.H) / cam.H, O.max_threads()


def cpu_baseline(scene, cam, target, budget_s: float = 20.0):
    """The oracle's fwd+bwd of whole frames of the workload, repeated while within the
    budget (a per-call setup over all triangles makes a band of rows a poor sample)."""
    times, threads = [], 1
    while not times or (sum(times) < budget_s / 4 and len(times) < 3):
        dt, _, threads = oracle_sample(scene, cam, target, cam.H)
        times.append(dt)
    dt = float(np.median(times))
    return {"value": 1.0 / dt, "unit": "it/s", "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle fwd+bwd of the whole {cam.W}x{cam.H} frame, median of {len(times)} "
                      f"runs of {dt:.2f} s"}


def max_over_ranks(x: float, device: str) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's); `device`
    is where the process group's backend keeps tensors (cuda for NCCL, cpu for gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    if rank != 0:
        return
    scene, cam, target = make_workload()
    # a step is the oracle's fwd+bwd over a band of pixel rows of the workload's frame,
    # sized from one whole-frame warm-up so that the K steps take about two minutes
    t_frame, _, _ = oracle_sample(scene, cam, target, cam.H)
    rows = max(8, min(cam.H, int(cam.H * 120.0 / (max(args.steps, 1) * t_frame))))
    times, fracs, threads = [], [], 1
    for _ in range(args.steps):
        dt, frac, threads = oracle_sample(scene, cam, target, rows)
        times.append(dt)
        fracs.append(frac)
    its = sum(fracs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": its, "unit": "it/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / its, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_rows_per_step": rows},
            "cpu_baseline": {"value": its, "unit": "it/s", "cores": threads, "kind": "oracle",
                             "sample": f"{rows} of {cam.H} pixel rows of the {cam.W}x{cam.H} frame per step, fwd+bwd"},
            "e2e": {"value": its, "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
STAGES = ("preprocess", "bin_sort", "render_fwd", "render_bwd", "preprocess_bwd")   # render_fwd: with the L1 loss
# step_init, preprocess, bin_scan, bin_scatter, tile_sort, render_fwd, loss, render_bwd, preprocess_bwd
KERNELS_PER_STEP = 8


def run_sigmoid_step(args, dev, st, cam, imgs, grad, loss, tgt, dv, dsh, do, ds, capture, timed):
    """The headline step with the sigmoid window of Eq. indicator2 (graph replay)."""
    import torch
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import Context
    ctx_s = Context(dev)
    ctx_s.set_window(N.WINDOW_SIGMOID)
    ctx_s.preprocess(st, [cam])
    ctx_s.reserve(int(ctx_s.bin_sort(sync=True) * 1.25) + 1024)

    def step_sigmoid():
        ctx_s.preprocess(st, [cam])
        ctx_s.bin_sort(sync=False)
        ctx_s.render_fwd_l1(imgs, [tgt], [grad], loss)
        ctx_s.render_bwd([grad])
        ctx_s.preprocess_bwd(dv, dsh, do, ds)

    ctx_s.set_fragment_counting(True)
    step_sigmoid()
    info_s = ctx_s.check()
    ctx_s.set_fragment_counting(False)
    for _ in range(3):
        step_sigmoid()
    g_sig = capture(step_sigmoid)
    for _ in range(3):
        g_sig.replay()
    ev_sig = timed(g_sig, args.steps)
    torch.cuda.synchronize()
    n_pairs_s = int(ctx_s.check().n_pairs)
    sig_its = args.steps / (float(sum(a.elapsed_time(b) for a, b in ev_sig)) / 1000.0)
    sigmoid_line = {"it_per_s": round(sig_its, 2), "pairs": n_pairs_s,
                    "frag_composited": int(info_s.frag_composited),
                    "workload": "the same fwd+bwd step with the sigmoid window of Eq. indicator2"}
    del g_sig
    return sigmoid_line


def run_pixel_sort_step(args, dev, st, cam, imgs, grad, loss, tgt, dv, dsh, do, ds, capture, timed):
    """The headline step with the per-pixel sort (graph replay; the uncaptured warm-up
    sizes the candidate buffer), and its forward alone."""
    import torch
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import Context
    L = N.lib()
    ctx_p = Context(dev)
    ctx_p.set_sort(N.SORT_PIXEL)
    ctx_p.preprocess(st, [cam])
    ctx_p.reserve(int(ctx_p.bin_sort(sync=True) * 1.25) + 1024)

    def fwd_pixel():
        ctx_p.preprocess(st, [cam])
        ctx_p.bin_sort(sync=False)
        ctx_p.render_fwd(imgs)

    def step_pixel():
        fwd_pixel()
        N.check(L.tri_loss_l1(imgs[0].data_ptr(), tgt.data_ptr(), imgs[0].numel(), grad.data_ptr(),
                              loss.data_ptr(), int(torch.cuda.current_stream().cuda_stream)))
        ctx_p.render_bwd([grad])
        ctx_p.preprocess_bwd(dv, dsh, do, ds)

    for _ in range(3):
        step_pixel()
    torch.cuda.synchronize()
    g_step, g_fwd = capture(step_pixel), capture(fwd_pixel)
    for _ in range(3):
        g_step.replay()
        g_fwd.replay()
    ev_step = timed(g_step, args.steps)
    ev_fwd = timed(g_fwd, args.steps)
    torch.cuda.synchronize()
    info_p = ctx_p.check()
    its = args.steps / (float(sum(a.elapsed_time(b) for a, b in ev_step)) / 1000.0)
    fps = args.steps / (float(sum(a.elapsed_time(b) for a, b in ev_fwd)) / 1000.0)
    line = {"it_per_s": round(its, 2), "fwd_fps": round(fps, 2), "pairs": int(info_p.n_pairs),
            "workload": "the same fwd+bwd step with the per-pixel sort (fragments ordered by the depth of "
                        "their triangle's plane along each pixel's ray)"}
    del g_step, g_fwd
    return line


def run_ours(args, rank, world):
    import torch
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    scene, cam, target = make_workload()
    st = SceneTensors.from_numpy(scene)
    tgt = torch.as_tensor(target).cuda()
    ctx = Context(dev)
    ctx.preprocess(st, [cam])
    n_pairs = ctx.bin_sort(sync=True)
    ctx.reserve(int(n_pairs * 1.25) + 1024)
    imgs = new_images([cam])
    grad = torch.empty_like(imgs[0])
    loss = torch.empty((), device="cuda")
    dv, dsh = torch.empty_like(st.verts), torch.empty_like(st.sh)
    do, ds = torch.empty_like(st.opacity), torch.empty_like(st.sigma)

    def step(ev=None):
        if ev:
            ev[0].record()
        ctx.preprocess(st, [cam])
        if ev:
            ev[1].record()
        ctx.bin_sort(sync=False)
        if ev:
            ev[2].record()
        ctx.render_fwd_l1(imgs, [tgt], [grad], loss)     # the forward with the L1 loss fused
        if ev:
            ev[3].record()
        ctx.render_bwd([grad])
        if ev:
            ev[4].record()
        ctx.preprocess_bwd(dv, dsh, do, ds)
        if ev:
            ev[5].record()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MB > 129 MB L2
    for _ in range(args.warmup):
        step()
    info = ctx.check()
    # fragments of the workload: per pixel, its last composited list entry + 1; and the
    # forward's own counts of evaluated and composited entries (one counted forward)
    t_fin = [torch.empty((cam.H, cam.W), device="cuda")]
    n_con = [torch.empty((cam.H, cam.W), device="cuda", dtype=torch.int32)]
    ctx.set_fragment_counting(True)
    ctx.preprocess(st, [cam])
    ctx.bin_sort(sync=False)
    ctx.render_fwd(imgs, t_fin, n_con)
    frags = int(n_con[0].sum(dtype=torch.int64).item())
    info_counted = ctx.check()
    ctx.set_fragment_counting(False)
    torch.cuda.synchronize()

    # the whole step as one CUDA graph (buffers are sized by the warm-up; capture allocates nothing)
    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def fwd_only():
        ctx.preprocess(st, [cam])
        ctx.bin_sort(sync=False)
        ctx.render_fwd(imgs)

    g_step = capture(step)
    # forward with the pruning statistics of Sec. 3.3 (largest T o, composited pixels)
    stat_w = torch.empty(st.n, device="cuda")
    stat_n = torch.empty(st.n, dtype=torch.int32, device="cuda")

    def fwd_stats():
        ctx.preprocess(st, [cam])
        ctx.bin_sort(sync=False)
        ctx.render_fwd(imgs, stats=(stat_w, stat_n))

    g_fwd = capture(fwd_only)
    g_fwd_stats = capture(fwd_stats)
    for _ in range(3):
        g_step.replay()
        g_fwd.replay()
        g_fwd_stats.replay()
    torch.cuda.synchronize()

    def timed(graph, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record()
            graph.replay()
            ev[k][1].record()
        return ev

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t_wall = time.perf_counter()
        ev_step = timed(g_step, args.steps)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    ev_fwd = timed(g_fwd, args.steps)
    ev_fwd_stats = timed(g_fwd_stats, args.steps)
    torch.cuda.synchronize()
    info = ctx.check()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev_step])
    total_ms = float(step_ms.sum())
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
    value = world * args.steps / (total_ms / 1000.0)
    fwd_ms = float(sum(a.elapsed_time(b) for a, b in ev_fwd))
    fps = args.steps / (fwd_ms / 1000.0)
    fps_stats = args.steps / (float(sum(a.elapsed_time(b) for a, b in ev_fwd_stats)) / 1000.0)

    # per-stage breakdown: eager steps with events between the calls (same stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    stage_ms = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(len(STAGES))]
                         for k in range(args.steps)])

    # end to end through the C ABI with host buffers: every step copies its scene and
    # target in from pinned host memory and its loss and parameter gradients back out.
    # Two device buffer sets (one captured step graph each) let step k + 1's copy-in and
    # step k's copy-out (separate copy streams, one per direction) overlap the compute.
    host = {k: v.cpu().pin_memory() for k, v in (("verts", st.verts), ("sh", st.sh), ("opacity", st.opacity),
                                                  ("sigma", st.sigma), ("target", tgt))}
    hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in
            (("dv", dv), ("dsh", dsh), ("do", do), ("ds", ds), ("loss", loss))}
    h2d = sum(v.numel() * 4 for v in host.values())
    d2h = sum(v.numel() * 4 for v in hout.values())

    def buffer_set():
        b = {"st": SceneTensors(torch.empty_like(st.verts), torch.empty_like(st.sh), torch.empty_like(st.opacity),
                                torch.empty_like(st.sigma), st.sh_degree),
             "tgt": torch.empty_like(tgt), "loss": torch.empty((), device="cuda"),
             "g": [torch.empty_like(x) for x in (dv, dsh, do, ds)]}
        for k in ("verts", "sh", "opacity", "sigma"):
            getattr(b["st"], k).copy_(getattr(st, k))
        b["tgt"].copy_(tgt)

        def fn():
            ctx.preprocess(b["st"], [cam])
            ctx.bin_sort(sync=False)
            ctx.render_fwd_l1(imgs, [b["tgt"]], [grad], b["loss"])
            ctx.render_bwd([grad])
            ctx.preprocess_bwd(*b["g"])
        fn()
        torch.cuda.synchronize()
        b["graph"] = capture(fn)
        return b

    sets = [buffer_set(), buffer_set()]
    cs, up, down = torch.cuda.current_stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    inputs_free = [ev(), ev()]     # the step that read a set's inputs has finished
    outputs_free = [ev(), ev()]    # a set's gradients have been copied out
    for e in inputs_free + outputs_free:
        e.record(cs)

    def e2e_step(k):
        b = sets[k % 2]
        with torch.cuda.stream(up):
            up.wait_event(inputs_free[k % 2])
            for key in ("verts", "sh", "opacity", "sigma"):
                getattr(b["st"], key).copy_(host[key], non_blocking=True)
            b["tgt"].copy_(host["target"], non_blocking=True)
            copied_in = torch.cuda.Event()
            copied_in.record(up)
        cs.wait_event(copied_in)
        cs.wait_event(outputs_free[k % 2])
        b["graph"].replay()
        inputs_free[k % 2].record(cs)
        with torch.cuda.stream(down):
            down.wait_event(inputs_free[k % 2])
            for key, x in zip(("dv", "dsh", "do", "ds"), b["g"]):
                hout[key].copy_(x, non_blocking=True)
            hout["loss"].copy_(b["loss"], non_blocking=True)
            outputs_free[k % 2].record(down)

    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    up.wait_event(e0)
    down.wait_event(e0)
    for k in range(args.steps):
        e2e_step(k)
    cs.wait_event(outputs_free[(args.steps - 1) % 2])
    e1.record(cs)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    # the host link's rate for the same copies (in alone, out alone, both at once)
    b0 = sets[0]

    def copy_in():
        with torch.cuda.stream(up):
            for key in ("verts", "sh", "opacity", "sigma"):
                getattr(b0["st"], key).copy_(host[key], non_blocking=True)
            b0["tgt"].copy_(host["target"], non_blocking=True)

    def copy_out():
        with torch.cuda.stream(down):
            for key, x in zip(("dv", "dsh", "do", "ds"), b0["g"]):
                hout[key].copy_(x, non_blocking=True)
            hout["loss"].copy_(b0["loss"], non_blocking=True)

    def link_gbs(fn, nbytes, reps=10):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return nbytes * reps / (time.perf_counter() - t0) / 1e9

    link = {"h2d_gbs": link_gbs(copy_in, h2d), "d2h_gbs": link_gbs(copy_out, d2h),
            "both_gbs": link_gbs(lambda: (copy_in(), copy_out()), h2d + d2h)}
    del sets, b0
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, "cuda")
    # the same step with the sigmoid window (Eq. indicator2): supports beyond the triangles
    sigmoid_line = None
    if not args.no_sigmoid:
        sigmoid_line = run_sigmoid_step(args, dev, st, cam, imgs, grad, loss, tgt, dv, dsh, do, ds, capture, timed)
    pixel_sort_line = None
    if not args.no_pixel_sort:
        pixel_sort_line = run_pixel_sort_step(args, dev, st, cam, imgs, grad, loss, tgt, dv, dsh, do, ds, capture,
                                              timed)

    e2e = {"value": world * args.steps / (e2e_ms / 1000.0), "unit": "it/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}
    # the copies' rate in the timed steps against the link's own with both directions busy
    e2e_gbs = (h2d + d2h) * args.steps / (e2e_ms / 1000.0) / 1e9
    e2e["link"] = {"achieved_gbs": round(e2e_gbs, 1), **{k: round(v, 1) for k, v in link.items()},
                   "frac_of_both": round(e2e_gbs / link["both_gbs"], 3),
                   "note": "pinned host <-> HBM copies of the step's inputs and outputs, timed alone"}

    if rank != 0:
        return
    clocks = clk.summary()
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    med = np.median(stage_ms, axis=0)
    # (stage times are eager; the graph removes launch gaps, not kernel time)
    breakdown = {s: round(float(m), 4) for s, m in zip(STAGES, med)}
    dom = STAGES[int(np.argmax(med))]
    # roofline of the dominant stage: fragments x ops per fragment on each pipe over the
    # stage time, against that pipe's peak at the measured maximum clock; the binding
    # pipe is the one with the largest fraction
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    F_eval, F_kept = int(info_counted.frag_evaluated), int(info_counted.frag_composited)

    def pipe_roofline(kernel):
        """The method's work (ENTRY_OPS per entry up to termination, COMPOSITED_OPS per
        composited fragment) over the stage time, per pipe against that pipe's peak at
        the measured maximum clock; the binding pipe is the one with the larger
        fraction."""
        t = med[STAGES.index(kernel)] / 1e3
        best = None
        for pipe, lanes in (("fma", FP32_LANES_PER_SM), ("mufu", MUFU_PER_SM)):
            peak = sms * lanes * clock_mhz * 1e6 / 1e12
            ops = frags * ENTRY_OPS[pipe] + F_kept * COMPOSITED_OPS[kernel][pipe]
            ach = ops / t / 1e12
            dense = frags * DENSE_FRAG_OPS[kernel][pipe] / t / 1e12
            if best is None or ach / peak > best["frac"]:
                best = {"bound": "alu", "kernel": kernel, "pipe": pipe, "achieved": round(ach, 3),
                        "peak": round(peak, 3), "unit": f"T {pipe.upper()} ops/s", "frac": round(ach / peak, 4),
                        "units": {"entries": frags, "composited": F_kept},
                        "unit_of_work": "entry (pixel x tile-list entry up to the pixel's termination) and "
                                        "composited fragment (alpha >= 1/255)",
                        "ops_per_unit": {"entry": ENTRY_OPS[pipe], "composited": COMPOSITED_OPS[kernel][pipe]},
                        "time_ms": round(t * 1e3, 4),
                        "frac_dense_equiv": round(dense / peak, 4),
                        "frac_dense_equiv_note": f"every entry charged {DENSE_FRAG_OPS[kernel][pipe]} ops: an "
                                                 "effective rate, not a fraction of executed work",
                        "peak_source": f"{sms} SMs x {lanes} lanes x {clock_mhz:.0f} MHz ({peak_src} max clock)"}
        best["traffic"] = _profiled_traffic(kernel + "_kernel")
        best["traffic_unit"] = "DRAM bytes per launch (ncu)"
        return best

    if dom in ("render_fwd", "render_bwd"):
        roof = pipe_roofline(dom)
    else:
        hbm = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None}
    roof_fwd = pipe_roofline("render_fwd")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "it/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "triangles": int(st.n), "width": cam.W, "height": cam.H, "views": 1,
                   "sh_degree": 3, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "fwd_fps": round(fps, 2),
        "fwd_fps_with_prune_stats": round(fps_stats, 2),
        "sigmoid_window": sigmoid_line,
        "per_pixel_sort": pixel_sort_line,
        "timing": "CUDA-graph replay of the whole step per timed iteration; stage_ms_median from eager "
                  "steps with events between the calls",
        "stage_ms_median": breakdown,
        "stage_hbm": stage_gbs(stage_bytes(int(st.n), 1, int(info.n_visible), int(info.n_pairs), cam.W * cam.H),
                               breakdown, float(peaks["hbm_gbs"])),
        "workload_stats": {"pairs": int(info.n_pairs), "visible": int(info.n_visible),
                           "frag_evaluated": F_eval, "frag_composited": F_kept},
        "roofline": roof,
        "roofline_render_fwd": roof_fwd,
        "e2e": e2e,
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clocks,
        "wall_s_timed": round(t_wall, 4),
    }
    if not args.no_multiview and world == 1:
        del g_step, g_fwd, g_fwd_stats
        line["multiview_3m_16views"] = run_multiview(max(3, min(args.steps, 10)), 3)
    if not args.no_densify and world == 1:
        line["densify_3m"] = run_densify(max(3, min(args.steps, 20)))
    if not args.no_solid and world == 1:
        line["solid_2m"] = run_solid(max(3, min(args.steps, 20)))
    if not args.no_noalloc and world == 1:
        line["noalloc_60k"] = run_noalloc(max(3, min(args.steps, 50)))
    if not args.no_serving:
        line["serving"] = run_serving(args.serve_requests, 2000.0, 1_000_000)
    if not args.no_multiscene and world == 1:
        line["multiscene_serving"] = run_multiscene(args.serve_requests)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(scene, cam, target, args.cpu_budget)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# multi-view training step: 3M triangles on 16 shells, 16 ring views at 1558x1038
# ---------------------------------------------------------------------------------------
def run_multiview(steps: int, warmup: int, n_tris: int = 3_000_000, n_views: int = 16):
    """fwd+bwd over all views per step, cameras re-drawn every step (seeded ring offset);
    eager calls, since the cameras change between steps. Returns a dict for the JSON line."""
    import torch
    from paper_2505_19175_gb300 import synth
    from paper_2505_19175_gb300.renderer import Context, SceneTensors
    st = SceneTensors.from_numpy(synth.scene_shells(n_tris, seed=1003))
    rng = np.random.default_rng(1003)
    offsets = rng.uniform(0.0, 2 * np.pi / n_views, warmup + 2 * steps + 1)
    W, H = 1558, 1038
    cams0 = synth.ring_cameras(n_views, W=W, H=H, offset=float(offsets[0]))
    imgs = torch.empty((n_views, 3, H, W), device="cuda")
    grad = torch.empty_like(imgs)
    tgt = torch.as_tensor(np.random.default_rng(1003).random((n_views, 3, H, W), dtype=np.float32)).cuda()
    loss = torch.empty((), device="cuda")
    dv, dsh = torch.empty_like(st.verts), torch.empty_like(st.sh)
    do, ds = torch.empty_like(st.opacity), torch.empty_like(st.sigma)
    ctx = Context()
    ctx.preprocess(st, cams0)
    ctx.reserve(int(ctx.bin_sort(sync=True) * 1.5) + 4096)
    views = [imgs[v] for v in range(n_views)]
    grads = [grad[v] for v in range(n_views)]
    tgts = [tgt[v] for v in range(n_views)]

    def step(k, fwd_only=False, ev=None):
        cams = synth.ring_cameras(n_views, W=W, H=H, offset=float(offsets[k]))
        if ev:
            ev[0].record()
        ctx.preprocess(st, cams)
        if ev:
            ev[1].record()
        ctx.bin_sort(sync=False)
        if ev:
            ev[2].record()
        if fwd_only:
            ctx.render_fwd(views)
            return
        ctx.render_fwd_l1(views, tgts, grads, loss)
        if ev:
            ev[3].record()
        ctx.render_bwd(grads)
        if ev:
            ev[4].record()
        ctx.preprocess_bwd(dv, dsh, do, ds)
        if ev:
            ev[5].record()

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()

    def timed(k0, fwd_only):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            ev[i][0].record()
            step(k0 + i, fwd_only)
            ev[i][1].record()
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in ev])

    ms = timed(warmup, False)
    info = ctx.check()
    ms_fwd = timed(warmup + steps, True)
    info_f = ctx.check()
    # per stage: the same steps with events between the calls (same stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(steps)]
    for i in range(steps):
        step(warmup + i, ev=evs[i])
    torch.cuda.synchronize()
    info_s = ctx.check()
    stage_ms = np.array([[evs[i][j].elapsed_time(evs[i][j + 1]) for j in range(len(STAGES))] for i in range(steps)])
    med = {k: round(float(v), 4) for k, v in zip(STAGES, np.median(stage_ms, axis=0))}
    ctx.set_fragment_counting(True)
    step(warmup + 2 * steps)
    info = ctx.check()
    ctx.set_fragment_counting(False)
    peaks, _ = _peaks()
    hbm = float(peaks["hbm_gbs"])
    nb = stage_bytes(n_tris, n_views, int(info_s.n_visible), int(info_s.n_pairs), n_views * W * H)
    return {"workload": f"{n_tris} tris SH3 on 16 shells, {n_views} ring views {W}x{H} per step, ring offset "
                        "re-drawn every step, fwd+bwd with L1 loss; params 708 MB > L2",
            "it_per_s": round(1000.0 * steps / float(ms.sum()), 3), "ms_per_step_median": round(float(np.median(ms)), 3),
            "views_per_s": round(1000.0 * steps * n_views / float(ms.sum()), 2),
            "fwd_fps_per_view": round(1000.0 * steps * n_views / float(ms_fwd.sum()), 2),
            "stage_ms_median": med,
            "sort_share": round(med["bin_sort"] / sum(med.values()), 4),
            "stage_hbm": stage_gbs(nb, med, hbm),
            "pairs": int(info.n_pairs), "visible_items": int(info.n_visible),
            "frag_evaluated": int(info.frag_evaluated), "frag_composited": int(info.frag_composited),
            "overflow": bool(info.overflow or info_f.overflow), "steps": steps, "warmup": warmup,
            "timing": "eager calls, CUDA events per step; stage_ms_median from steps with events between the "
                      "calls; stage_hbm = algorithmic bytes (stage_bytes) over the stage time, against the "
                      "measured HBM copy rate"}


# ---------------------------------------------------------------------------------------
# opaque-triangle render of a 2M-triangle soup at 720p / 1080p / 4k
# ---------------------------------------------------------------------------------------
def run_solid(steps: int, n_tris: int = 2_000_000):
    import torch
    from paper_2505_19175_gb300 import synth
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    st = SceneTensors.from_numpy(synth.scene_shells(n_tris, seed=1005))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": f"{n_tris} tris SH3 on 16 shells, opaque render (sigma -> 0, o = 1 limit), camera at "
                       "radius 4 looking at the centre; CUDA-graph replay of preprocess + binning + render; "
                       "L2 flushed between frames"}
    for W, H in ((1280, 720), (1920, 1080), (3840, 2160)):
        cam = synth.ring_cameras(1, W=W, H=H)[0]
        ctx = Context()
        imgs = new_images([cam])
        ids = [torch.empty((H, W), dtype=torch.int32, device="cuda")]
        pairs = ctx.render_solid(st, [cam], imgs, ids, sync_pairs=True)
        ctx.reserve(int(pairs * 1.25) + 1024)
        for _ in range(3):
            ctx.render_solid(st, [cam], imgs, ids, sync_pairs=False)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.render_solid(st, [cam], imgs, ids, sync_pairs=False)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record()
            g.replay()
            ev[k][1].record()
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        info = ctx.check()
        out[f"{W}x{H}"] = {"fps": round(1000.0 * steps / float(ms.sum()), 1),
                           "ms_median": round(float(np.median(ms)), 4), "pairs": int(info.n_pairs),
                           "visible": int(info.n_visible), "overflow": bool(info.overflow)}
        del g
    return out


# ---------------------------------------------------------------------------------------
# the allocation-free forward (its own fixed workspace; preprocess, onesweep radix sort
# of the 64-bit tile|depth keys, render) against the regular entry points on one scene
# ---------------------------------------------------------------------------------------
def run_noalloc(steps: int, n_tris: int = 60_000):
    import ctypes as C
    import torch
    from paper_2505_19175_gb300 import native as N, synth
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    scene, _, _ = synth.scene_patches(n=n_tris, n_patch=40)
    cam = synth.camera_patches()
    st = SceneTensors.from_numpy(scene)
    f = N.lib().tri_render_fwd_noalloc
    f.argtypes = [C.POINTER(N.tri_scene), C.POINTER(N.tri_camera), C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    img = torch.empty((3, cam.H, cam.W), device="cuda")
    T = torch.empty((cam.H, cam.W), device="cuda")
    nc = torch.empty((cam.H, cam.W), device="cuda", dtype=torch.int32)
    status = torch.zeros((1,), device="cuda", dtype=torch.int32)
    abi_scene, abi_cam = st.as_abi(), N.make_camera(cam)
    stream = int(torch.cuda.current_stream().cuda_stream)

    def noalloc():
        if f(C.byref(abi_scene), C.byref(abi_cam), img.data_ptr(), T.data_ptr(), nc.data_ptr(),
             status.data_ptr(), stream) != 0:
            raise RuntimeError("tri_render_fwd_noalloc failed")

    ctx = Context()
    imgs = new_images([cam])

    def regular():
        ctx.preprocess(st, [cam])
        ctx.bin_sort(sync=False)
        ctx.render_fwd(imgs)

    ctx.preprocess(st, [cam])
    ctx.reserve(int(ctx.bin_sort(sync=True) * 1.25) + 1024)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": f"{n_tris} tris SH3 on 40 planar patches, 1297x840, forward only, eager calls, "
                       "L2 flushed between frames"}
    for name, fn in (("noalloc", noalloc), ("regular", regular)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record()
            fn()
            ev[k][1].record()
        torch.cuda.synchronize()
        out[name + "_ms_median"] = round(float(np.median([a.elapsed_time(b) for a, b in ev])), 4)
    out["status"] = int(status.item())
    out["pairs"] = int(ctx.check().n_pairs)
    return out


# ---------------------------------------------------------------------------------------
# densification moves and the size regulariser on 3M triangles
# ---------------------------------------------------------------------------------------
def run_densify(steps: int, n: int = 3_000_000, frac: float = 0.1):
    import torch
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import Context
    g = torch.Generator(device="cuda").manual_seed(1006)
    k = int(n * frac)
    cap = n + 3 * k
    v0 = torch.randn((cap, 3, 3), device="cuda", generator=g) * 0.1
    sh0 = torch.randn((cap, 16, 3), device="cuda", generator=g) * 0.2
    o0 = torch.rand(cap, device="cuda", generator=g)
    s0 = torch.rand(cap, device="cuda", generator=g) + 0.3
    sel = torch.randperm(n, device="cuda", generator=g)[:k].to(torch.int32)
    noise = torch.randn((k, 2), device="cuda", generator=g)
    e1, e2 = v0[:n, 1] - v0[:n, 0], v0[:n, 2] - v0[:n, 0]
    tau = float(0.5 * torch.linalg.cross(e1, e2).norm(dim=1).median())
    ctx = Context()
    n_out = torch.empty(1, dtype=torch.int64, device="cuda")
    bufs = [x.clone() for x in (v0, sh0, o0, s0)]
    st = torch.cuda.current_stream().cuda_stream
    L = N.lib()

    def once():
        for b_, x in zip(bufs, (v0, sh0, o0, s0)):
            b_[:n].copy_(x[:n])
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        N.check(L.tri_densify(ctx.h, bufs[0].data_ptr(), bufs[1].data_ptr(), bufs[2].data_ptr(), bufs[3].data_ptr(),
                              3, n, cap, sel.data_ptr(), k, noise.data_ptr(), 0.01, tau, n_out.data_ptr(), st))
        ev[1].record()
        return ev

    for _ in range(2):
        once()
    evs = [once() for _ in range(steps)]
    torch.cuda.synchronize()
    dms = float(np.median([a.elapsed_time(b) for a, b in evs]))
    grad = torch.zeros_like(v0[:n])
    loss = torch.empty((), device="cuda")
    rev = []
    for _ in range(steps + 2):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        N.check(L.tri_size_reg(v0.data_ptr(), n, 1.0 / n, loss.data_ptr(), grad.data_ptr(), st))
        ev[1].record()
        rev.append(ev)
    torch.cuda.synchronize()
    rms = float(np.median([a.elapsed_time(b) for a, b in rev[2:]]))
    added = int(n_out.item()) - n
    # bytes: densify reads 236 B and writes 236 B per selected triangle plus 236 B per
    # appended one; the regulariser reads 36 B and read-modify-writes 36 B of gradient
    dens_bytes = k * 472 + added * 236
    reg_bytes = n * 108
    return {"workload": f"{n} tris SH3, {k} selected (tau_small = median area: about half split, half cloned)",
            "densify_ms": round(dms, 4), "appended": added,
            "densify_gbs": round(dens_bytes / (dms * 1e-3) / 1e9, 1),
            "size_reg_ms": round(rms, 4), "size_reg_gbs": round(reg_bytes / (rms * 1e-3) / 1e9, 1)}


# ---------------------------------------------------------------------------------------
# serving: open-loop replay of a Poisson trace against one resident scene
# ---------------------------------------------------------------------------------------
def replay(srv, sid, trace, max_time_s=60.0):
    """Submit each request at its arrival time; returns wall seconds."""
    import torch
    free = {}
    pending = {}
    t0 = time.perf_counter()
    i = 0
    while i < len(trace) or pending:
        now = time.perf_counter() - t0
        while i < len(trace) and trace[i][0] <= now:
            cam = trace[i][2]
            key = (cam.H, cam.W)
            buf = free.get(key, [])
            out = buf.pop() if buf else torch.empty((3, cam.H, cam.W), device="cuda")
            t, _ = srv.submit(sid, cam, out)
            pending[t] = (key, out)
            i += 1
        for t, _st in srv.poll():
            key, out = pending.pop(t)
            free.setdefault(key, []).append(out)
        if now > max_time_s:
            break
        time.sleep(0.0001)
    return time.perf_counter() - t0


def serve_trace(scene, trace, warm_rate: float, **kw) -> dict:
    """One server over one open-loop trace (after a warm-up trace of the same mix that
    grows the workspaces and captures the graphs); its latency and throughput stats."""
    import torch
    from paper_2505_19175_gb300 import synth
    from paper_2505_19175_gb300.serve import Server
    srv = Server(max_width=1920, max_height=1080, use_graphs=True, **kw)
    sid = srv.add_scene(scene)
    replay(srv, sid, synth.serve_requests(512, seed=999, rate_hz=warm_rate))
    torch.cuda.synchronize()
    srv.reset_stats()
    wall = replay(srv, sid, trace)
    st = srv.stats()
    srv.close()
    return {"p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
            "max_ms": round(st["max_ms"], 3), "fps": round(st["fps"], 1),
            "completed": int(st["completed"]), "mean_batch": round(st["mean_batch"], 2),
            "queue_p99_ms": round(st["queue_p99_ms"], 3), "graph_replays": int(st["graph_replays"]),
            "graph_captures": int(st["graph_captures"]), "eager_batches": int(st["eager_batches"]),
            "reruns": int(st["reruns"]), "reallocs": int(st["reallocs"]),
            "capture_ms": round(st["capture_ms"], 2), "eager_ms": round(st["eager_ms"], 2),
            "wall_s": round(wall, 3), **kw}


def run_serving(n_req: int, rate_hz: float, n_tris: int, saturation_rates=(2000.0, 8000.0, 20000.0)):
    from paper_2505_19175_gb300 import synth
    from paper_2505_19175_gb300.renderer import SceneTensors
    scene = SceneTensors.from_numpy(synth.scene_shells(n_tris, seed=1004))
    trace = synth.serve_requests(n_req, seed=1004, rate_hz=rate_hz)
    out = {"workload": f"{n_tris} tris SH3 shells, {n_req} requests, Poisson {rate_hz:.0f} req/s, "
                       "640x360 : 1280x720 : 1920x1080 = 2:2:1, open-loop"}
    for name, kw in (("batched", dict(max_batch=16, slots=4)), ("one_request_per_launch", dict(max_batch=1, slots=1))):
        out[name] = serve_trace(scene, trace, rate_hz, **kw)
    # continuous batching against one request per launch at equal concurrency (4 slots,
    # each its own stream), at the arrival rate above and at rates beyond what one
    # request per launch sustains; the same trace shape (seed) at each rate
    sat = {"note": "same Poisson trace seed at each rate; both arms 4 slots; fps = completed / wall"}
    for r in saturation_rates:
        tr = synth.serve_requests(n_req, seed=1004, rate_hz=r)
        sat[f"{r:.0f}_req_s"] = {name: serve_trace(scene, tr, r, **kw) for name, kw in
                                 (("batched", dict(max_batch=16, slots=4)),
                                  ("unbatched", dict(max_batch=1, slots=4)))}
    out["equal_slots"] = sat
    return out


# ---------------------------------------------------------------------------------------
# multi-scene serving under a memory budget with a concurrent training job
# ---------------------------------------------------------------------------------------
def run_multiscene(n_req: int, rate_hz: float = 2000.0, budget_gb: float = 60.0):
    """8 resident scenes (N log-uniform in [200k, 2M]) served from one budget while a
    fwd+bwd training job of 8 views at 1297x840 runs on scene 0 on its own stream."""
    import threading
    import torch
    from paper_2505_19175_gb300 import synth
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    from paper_2505_19175_gb300.serve import Server
    sizes = synth.scene_sizes_multi()
    scenes = [synth.scene_shells(n, seed=2000 + i) for i, n in enumerate(sizes)]
    srv = Server(mem_budget_bytes=int(budget_gb * (1 << 30)), max_batch=16, slots=4, max_width=1920, max_height=1080)
    sids = [srv.add_scene(sc) for sc in scenes]
    trace = synth.serve_requests(n_req, seed=1007, rate_hz=rate_hz, n_scenes=len(scenes))
    warm = synth.serve_requests(512, seed=998, rate_hz=rate_hz, n_scenes=len(scenes))

    # training job on scene 0
    st = SceneTensors.from_numpy(scenes[0])
    cams = synth.ring_cameras(8, W=1297, H=840)
    tstream = torch.cuda.Stream()
    ctx = Context()
    imgs = new_images(cams)
    grads = [torch.empty_like(x) for x in imgs]
    tgt = [torch.rand_like(x) for x in imgs]
    loss = torch.empty((), device="cuda")
    dv, dsh = torch.empty_like(st.verts), torch.empty_like(st.sh)
    do, ds = torch.empty_like(st.opacity), torch.empty_like(st.sigma)
    with torch.cuda.stream(tstream):
        ctx.preprocess(st, cams, stream=tstream)
        ctx.reserve(int(ctx.bin_sort(sync=True, stream=tstream) * 1.25) + 4096)

    def train_step():
        ctx.preprocess(st, cams, stream=tstream)
        ctx.bin_sort(sync=False, stream=tstream)
        ctx.render_fwd_l1(imgs, [tgt[v] for v in range(len(cams))], grads, loss, stream=tstream)
        ctx.render_bwd(grads, stream=tstream)
        ctx.preprocess_bwd(dv, dsh, do, ds, stream=tstream)

    def train_for(seconds: float):
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            train_step()
            tstream.synchronize()
            n += 1
        return n / (time.perf_counter() - t0)

    for _ in range(3):
        train_step()
    tstream.synchronize()
    alone = train_for(1.0)

    # serving with per-request latencies measured at poll (host clock)
    def replay_lat(tr, max_time_s=60.0):
        free, pending, lat = {}, {}, []
        t0 = time.perf_counter()
        i = 0
        while i < len(tr) or pending:
            now = time.perf_counter() - t0
            while i < len(tr) and tr[i][0] <= now:
                _, sc, cam = tr[i]
                key = (cam.H, cam.W)
                buf = free.get(key, [])
                out = buf.pop() if buf else torch.empty((3, cam.H, cam.W), device="cuda")
                t, _ = srv.submit(sids[sc], cam, out)
                pending[t] = (key, out, sc, time.perf_counter())
                i += 1
            for t, status in srv.poll():
                key, out, sc, ts = pending.pop(t)
                lat.append((sc, (time.perf_counter() - ts) * 1e3, status))
                free.setdefault(key, []).append(out)
            if now > max_time_s:
                break
            time.sleep(0.0001)
        return lat, time.perf_counter() - t0

    replay_lat(warm)
    torch.cuda.synchronize()
    stop = threading.Event()
    steps = [0]

    def trainer():
        while not stop.is_set():
            train_step()
            tstream.synchronize()
            steps[0] += 1

    th = threading.Thread(target=trainer)
    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(0.0002)      # the submit / poll loop and the trainer share the GIL
    t_start = time.perf_counter()
    th.start()
    lat, wall = replay_lat(trace)
    stop.set()
    th.join()
    sys.setswitchinterval(old_switch)
    t_train = time.perf_counter() - t_start
    stats = srv.stats()
    srv.close()
    per_scene = []
    for k, n in enumerate(sizes):
        ms = np.array([x[1] for x in lat if x[0] == k and x[2] == 0])
        per_scene.append({"triangles": n, "completed": int(len(ms)),
                          "p50_ms": round(float(np.percentile(ms, 50)), 3) if len(ms) else None,
                          "p99_ms": round(float(np.percentile(ms, 99)), 3) if len(ms) else None})
    return {"workload": f"{len(sizes)} shell scenes, {sum(sizes)} tris SH3 resident under a {budget_gb:.0f} GB budget; "
                        f"{n_req} requests Poisson {rate_hz:.0f} req/s over the scenes, 640x360 : 1280x720 : 1920x1080 "
                        "= 2:2:1; concurrently a fwd+bwd job of 8 views at 1297x840 on scene 0 on its own stream",
            "per_scene": per_scene, "serving_fps": round(stats["fps"], 1), "rejected": int(stats["rejected"]),
            "bytes_resident": int(stats["bytes_resident"]), "training_it_per_s": round(steps[0] / t_train, 2),
            "training_it_per_s_alone": round(alone, 2), "wall_s": round(wall, 3),
            "latency": "host clock from submit to poll (0.1 ms polling)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-multiview", action="store_true")
    ap.add_argument("--no-solid", action="store_true")
    ap.add_argument("--no-densify", action="store_true")
    ap.add_argument("--no-sigmoid", action="store_true")
    ap.add_argument("--no-pixel-sort", action="store_true")
    ap.add_argument("--no-multiscene", action="store_true")
    ap.add_argument("--no-noalloc", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=4096)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
