"""The per-pixel sort variant on the GPU against the oracle in the same mode (each
pixel's fragments by the depth of their triangle's plane along its ray): images
within 1e-4 and composited counts equal on the pixels FP32 resolves, the others equal
to one of the oracle's listed outcomes, gradients within 1e-3; and on crossing triangles the GPU result differs from the tile sort exactly where
the oracle's does."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth
from gpu_util import check_image
from test_gpu_backward import _check_grads, _masked_grad
from test_oracle_render import one_tri_scene, stack

pytestmark = pytest.mark.gpu
PIXEL = dict(O.DEFAULT_CONSTS, sort=O.SORT_PIXEL)


def _forward(scene, cams, sort=1):
    import torch
    from paper_2505_19175_gb300.renderer import Context, SceneTensors, new_images
    st = SceneTensors.from_numpy(scene)
    ctx = Context()
    ctx.set_sort(sort)
    ctx.preprocess(st, cams)
    ctx.bin_sort(sync=True)
    imgs = new_images(cams)
    T = [torch.empty((c.H, c.W), device="cuda") for c in cams]
    nc = [torch.empty((c.H, c.W), device="cuda", dtype=torch.int32) for c in cams]
    ctx.render_fwd(imgs, T, nc)
    ctx.check()
    torch.cuda.synchronize()
    return ([x.cpu().numpy().astype(np.float64) for x in imgs], [x.cpu().numpy() for x in T],
            [x.cpu().numpy() for x in nc], ctx, st)


def _compare(img, T, nc, ref, label):
    check_image(img, T.astype(np.float64), ref, label=label, n_kept=nc)


@pytest.mark.parametrize("seed,W,H", [(81, 96, 80), (82, 61, 37)])
def test_per_pixel_sort_forward_matches_oracle(seed, W, H):
    # random orientations: many triangles intersect, so pixel and centroid orders differ
    scene = synth.random_scene(400, seed=seed, deg=2, size=(0.1, 0.8), sigma=(0.4, 3.0), opacity=(0.05, 0.9))
    cam = synth.camera_identity(W, H)
    imgs, T, nc, _, _ = _forward(scene, [cam])
    ref = O.render(scene, cam, PIXEL, flags=True)
    _compare(imgs[0], T[0], nc[0], ref, f"per-pixel sort {W}x{H}")
    tile = O.render(scene, cam)
    assert np.abs(tile["image"] - ref["image"]).max() > 1e-2     # the orders really differ


def test_crossing_triangles_follow_the_nearer_plane():
    cam = synth.camera_identity(64, 48, fx=50.0)
    s = stack(one_tri_scene(cam, np.array([[4.0, 4.0], [60.0, 8.0], [20.0, 44.0]]), np.array([2.0, 6.0, 5.0]),
                            rgb=(0.9, 0.1, 0.2), o=0.7, sigma=1.3),
              one_tri_scene(cam, np.array([[58.0, 42.0], [6.0, 30.0], [50.0, 3.0]]), np.full(3, 4.0),
                            rgb=(0.1, 0.3, 0.8), o=0.6, sigma=0.8))
    s = synth.Scene(s["verts"].astype(np.float32), s["sh"].astype(np.float32), s["opacity"].astype(np.float32),
                    s["sigma"].astype(np.float32), 0)
    imgs, T, nc, _, _ = _forward(s, [cam])
    ref = O.render(s, cam, PIXEL, flags=True)
    _compare(imgs[0], T[0], nc[0], ref, "crossing triangles")
    tile_gpu = _forward(s, [cam], sort=0)[0][0]
    tile_ref = O.render(s, cam)["image"]
    ok = ref["flags"] == 0
    want = np.abs(tile_ref - ref["image"]).max(0) > 1e-3
    got = np.abs(tile_gpu - imgs[0]).max(0) > 1e-3
    assert want[ok].sum() > 50
    np.testing.assert_array_equal(got[ok], want[ok])


def test_per_pixel_sort_two_views():
    scene = synth.random_scene(300, seed=83, deg=1, size=(0.1, 0.6))
    cams = [synth.camera_look_at((0.2 * k - 0.1, 0.0, -0.3), (0, 0, 3.5), 72, 56) for k in range(2)]
    imgs, T, nc, _, _ = _forward(scene, cams)
    for k, c in enumerate(cams):
        _compare(imgs[k], T[k], nc[k], O.render(scene, c, PIXEL, flags=True), f"per-pixel sort view {k}")


def test_per_pixel_sort_backward_matches_oracle():
    from gpu_util import gpu_backward
    scene = synth.random_scene(300, seed=84, deg=2, size=(0.1, 0.7), sigma=(0.5, 2.5), opacity=(0.05, 0.9))
    cam = synth.camera_identity(80, 64)
    imgs, T, nc, ctx, st = _forward(scene, [cam])
    ref = O.render(scene, cam, PIXEL, flags=True)
    g = _masked_grad(ref, 85, (3, cam.H, cam.W), "per-pixel sort")
    got = gpu_backward(ctx, st, [g])
    want = O.render_grad(scene, cam, g, PIXEL)
    _check_grads(got, want, label="per-pixel sort")
