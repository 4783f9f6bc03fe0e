"""The sigmoid window variant (Eq. indicator2) on the GPU against the oracle with the
same window: images within 1e-4 on the pixels FP32 resolves, tile lists of the
dilated supports against the oracle rectangles, gradients within 1e-3."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth
from gpu_util import check_image
from test_gpu_backward import _check_grads, _masked_grad

pytestmark = pytest.mark.gpu
SIG = dict(O.DEFAULT_CONSTS, window=O.WINDOW_SIGMOID)


def _forward(scene, cams):
    import torch
    from paper_2505_19175_gb300 import native as N
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    ctx.set_window(N.WINDOW_SIGMOID)
    ctx.preprocess(st, cams)
    ctx.bin_sort(sync=True)
    imgs = new_images(cams)
    T = [torch.empty((c.H, c.W), device="cuda") for c in cams]
    ctx.render_fwd(imgs, T)
    ctx.check()
    torch.cuda.synchronize()
    return [x.cpu().numpy().astype(np.float64) for x in imgs], [x.cpu().numpy() for x in T], ctx, st


@pytest.mark.parametrize("seed,W,H", [(71, 96, 80), (72, 61, 37)])
def test_sigmoid_forward_matches_oracle(seed, W, H):
    scene = synth.random_scene(150, seed=seed, deg=2, size=(0.05, 0.5), sigma=(0.3, 3.0), opacity=(0.02, 0.9))
    cam = synth.camera_identity(W, H)
    imgs, T, ctx, _ = _forward(scene, [cam])
    ref = O.render(scene, cam, SIG, flags=True)
    check_image(imgs[0], T[0].astype(np.float64), ref, label=f"sigmoid window {W}x{H}")
    # supports beyond the triangles: more pairs than with the paper's window
    info = O.tri_info(scene, cam, SIG)
    ot, oi = O.tile_pairs(scene, cam, SIG, info=info)
    amb = info["amb"] != 0
    tiles = ctx.debug("pair_tiles").astype(np.int64)
    items = ctx.debug("pair_items").astype(np.int64)
    assert {(t, i) for t, i in zip(tiles, items) if not amb[i]} == {(t, i) for t, i in zip(ot, oi) if not amb[i]}
    assert len(ot) > len(O.tile_pairs(scene, cam)[0])


def test_sigmoid_backward_matches_oracle():
    from gpu_util import gpu_backward
    scene = synth.random_scene(150, seed=73, deg=2, size=(0.05, 0.5), sigma=(0.4, 2.5), opacity=(0.05, 0.9))
    cam = synth.camera_identity(80, 64)
    imgs, T, ctx, st = _forward(scene, [cam])
    ref = O.render(scene, cam, SIG, flags=True)
    g = _masked_grad(ref, 74, (3, cam.H, cam.W), "sigmoid window")
    got = gpu_backward(ctx, st, [g])
    want = O.render_grad(scene, cam, g, SIG)
    _check_grads(got, want, label="sigmoid window")
