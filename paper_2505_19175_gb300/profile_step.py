"""A few eager fwd+bwd steps of one of the measured workloads, for running under a
profiler (each step: preprocess, tile binning and sort, forward with the L1 loss,
backward, preprocess backward, all through the C ABI).

    python -m paper_2505_19175_gb300.profile_step [--workload patches|shells] [--views N] [--steps K]
                                                  [--sort tile|pixel]

patches: 500,000 triangles on 200 planar patches, SH degree 3, one view at 1297x840.
shells: 3,000,000 triangles on 16 nested shells, SH degree 3, the first N of 16 ring
views at 1558x1038 (N = 16 is the training step of the benchmark; fewer views make a
smaller case for captures that replay a kernel many times). --sort pixel composites each
pixel's fragments in the order of their plane's depth along its ray (the per-pixel sort)
instead of the per-tile centroid order.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=("patches", "shells"), default="patches")
    ap.add_argument("--views", type=int, default=16, help="shells: number of ring views (1..16)")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--sort", choices=("tile", "pixel"), default="tile")
    args = ap.parse_args(argv)
    import torch
    from paper_2505_19175_gb300 import native, synth
    from paper_2505_19175_gb300.renderer import Context, SceneTensors

    if args.workload == "patches":
        scene, _, _ = synth.scene_patches()
        cams = [synth.camera_patches()]
    else:
        scene = synth.scene_shells(3_000_000, seed=1003)
        cams = synth.ring_cameras(16, W=1558, H=1038, offset=0.1)[:max(1, min(16, args.views))]
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    if args.sort == "pixel":
        ctx.set_sort(native.SORT_PIXEL)
    imgs = [torch.empty((3, c.H, c.W), device="cuda") for c in cams]
    grads = [torch.empty_like(x) for x in imgs]
    tgts = [torch.as_tensor(synth.target_image(c.H, c.W, seed=2002 + k)).cuda() for k, c in enumerate(cams)]
    loss = torch.empty((), device="cuda")
    dv, dsh = torch.empty_like(st.verts), torch.empty_like(st.sh)
    do, ds = torch.empty_like(st.opacity), torch.empty_like(st.sigma)
    for k in range(args.steps):
        ctx.preprocess(st, cams)
        ctx.bin_sort(sync=(k == 0))
        if args.sort == "pixel":
            # (the per-pixel sort's forward has no fused loss: the loss kernel follows it)
            ctx.render_fwd(imgs)
            for img, tgt, gr in zip(imgs, tgts, grads):
                native.check(native.lib().tri_loss_l1(img.data_ptr(), tgt.data_ptr(), img.numel(), gr.data_ptr(),
                                                      loss.data_ptr(), torch.cuda.current_stream().cuda_stream))
        else:
            ctx.render_fwd_l1(imgs, tgts, grads, loss)
        ctx.render_bwd(grads)
        ctx.preprocess_bwd(dv, dsh, do, ds)
    ctx.check()
    torch.cuda.synchronize()
    print(f"{args.workload}: {args.steps} steps over {len(cams)} view(s), {ctx.info().n_pairs} pairs")


if __name__ == "__main__":
    main()
