"""Parity at the measured workloads' full sizes, in the launch configuration the
benchmark times (one preprocess over every view, one tile sort, one render), checked on
seeded samples of pixels that the oracle evaluates one by one: images and T within
1e-4, and gradients within 1e-3 relative when dL/dimage is non-zero only on the sampled
pixels (so the oracle's adjoint over those pixels is the whole expected gradient)."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth
from gpu_util import gpu_backward, gpu_forward
from test_gpu_backward import _check_grads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-4


def _sample(cam, n, rng):
    mask = np.zeros((cam.H, cam.W), np.uint8)
    mask.reshape(-1)[rng.choice(cam.H * cam.W, n, replace=False)] = 1
    return mask


def _check_image(img, T, ref, mask):
    sel = mask.astype(bool)
    ok = sel & (ref["flags"] == 0)
    assert ok.sum() >= 0.99 * sel.sum()
    err = np.abs(img - ref["image"])[:, ok]
    assert err.max() <= TOL, err.max()
    assert np.abs(T - ref["T_final"])[ok].max() <= TOL
    return ok


def test_full_size_patch_backward_sampled_pixels():
    """500k triangles at 1297x840: gradients of 2,000 sampled pixels."""
    scene, _, _ = synth.scene_patches()
    cam = synth.camera_patches()
    imgs, T, nc, ctx, st = gpu_forward(scene, [cam])
    rng = np.random.default_rng(78)
    mask = _sample(cam, 2000, rng)
    mask[cam.H - 1, ::7] = 1        # ragged bottom row of tiles
    ref = O.render(scene, cam, pix_mask=mask, flags=True)
    ok = _check_image(imgs[0], T[0], ref, mask)
    g = (rng.standard_normal((3, cam.H, cam.W)) * ok[None]).astype(np.float32)
    got = gpu_backward(ctx, st, [g])
    want = O.render_grad(scene, cam, g, pix_mask=mask)
    assert (np.abs(want["opacity"]) > 0).sum() > 10_000      # many triangles take part
    _check_grads(got, want)


def test_full_size_shells_16_views_sampled_pixels():
    """3M triangles on nested shells, 16 ring views at 1558x1038 in one batch: two views
    checked on 1,500 sampled pixels each, and the gradient of those pixels summed over
    the two views (the other 14 views carry a zero dL/dimage)."""
    scene = synth.scene_shells()
    cams = synth.ring_cameras()
    imgs, T, nc, ctx, st = gpu_forward(scene, cams)
    rng = np.random.default_rng(79)
    dls = [np.zeros((3, c.H, c.W), np.float32) for c in cams]
    want = None
    for v in (0, 9):
        cam = cams[v]
        mask = _sample(cam, 1500, rng)
        ref = O.render(scene, cam, pix_mask=mask, flags=True)
        ok = _check_image(imgs[v], T[v], ref, mask)
        dls[v] = (rng.standard_normal((3, cam.H, cam.W)) * ok[None]).astype(np.float32)
        w = O.render_grad(scene, cam, dls[v], pix_mask=mask)
        want = w if want is None else {k: want[k] + w[k] for k in w}
    del imgs, T, nc
    got = gpu_backward(ctx, st, dls)
    _check_grads(got, want)
