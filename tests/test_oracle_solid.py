"""Pins of the oracle's solid-triangle render: the sigma -> 0, o = 1 limit of the splat
render (Sec. 5 turns the optimised soup into opaque triangles). Expected values come
from the window function (``O.window``) and from the pinned splat oracle in exact mode."""
import numpy as np

import oracle as O
from paper_2505_19175_gb300 import synth
from test_oracle_render import CAM, UV, one_tri_scene, pix_centres, stack


def _inside(uv, cam=CAM):
    ratio, _ = O.window(uv, 1.0, pix_centres(cam))
    return (ratio > 0).reshape(cam.H, cam.W)


def test_single_triangle_covers_exactly_its_interior():
    cam = synth.camera_identity(48, 40, fx=40.0)
    cam.bg = np.array([0.1, 0.0, 0.3], np.float32)
    rgb = np.array([0.7, 0.2, 0.4])
    s = one_tri_scene(cam, UV, np.array([3.0, 4.0, 5.0]), rgb=rgb, o=0.01, sigma=5.0)   # o, sigma ignored
    ref = O.render_solid(s, cam)
    inside = _inside(UV, cam)
    assert inside.sum() > 100
    np.testing.assert_array_equal(ref["id"], np.where(inside, 0, -1))
    want = np.where(inside[None], rgb[:, None, None], cam.bg.astype(float)[:, None, None])
    np.testing.assert_allclose(ref["image"], want, atol=1e-12)


def test_nearer_triangle_wins_the_overlap():
    uv_b = UV + [4.0, 3.0]
    near = one_tri_scene(CAM, UV, np.array([2.0, 2.0, 2.0]), rgb=(1.0, 0.0, 0.0))
    far = one_tri_scene(CAM, uv_b, np.array([6.0, 6.0, 6.0]), rgb=(0.0, 0.0, 1.0))
    for order in ((near, far), (far, near)):
        ids = O.render_solid(stack(*order), CAM)["id"]
        i_near = 0 if order[0] is near else 1
        a, b = _inside(UV), _inside(uv_b)
        np.testing.assert_array_equal(ids == i_near, a)
        np.testing.assert_array_equal(ids == 1 - i_near, b & ~a)


def test_equals_the_exact_mode_limit_of_the_splat_render():
    scene = synth.random_scene(400, seed=51, deg=1, size=(0.05, 0.6))
    cam = synth.camera_identity(80, 64)
    solid = O.render_solid(scene, cam)
    lim = dict(verts=scene.verts, sh=scene.sh, opacity=np.ones(scene.n), sigma=np.full(scene.n, 1e-9),
               sh_degree=scene.sh_degree)
    splat = O.render(lim, cam, consts=O.EXACT_CONSTS)
    # pixels whose winner is not within 1e-3 of its edge: the limit is reached to ~1e-8
    info = O.tri_info(scene, cam)
    ok = np.ones((cam.H, cam.W), bool)
    pts = pix_centres(cam)
    for t in np.unique(solid["id"][solid["id"] >= 0]):
        ratio, _ = O.window(info["q"][t], 1.0, pts)
        ok &= ~((solid["id"] == t) & (ratio.reshape(cam.H, cam.W) < 1e-3))
    ok &= solid["flags"] == 0
    assert ok.mean() > 0.9
    np.testing.assert_allclose(splat["image"][:, ok], solid["image"][:, ok], atol=1e-6)
    np.testing.assert_array_equal(splat["n_kept"][ok] > 0, solid["id"][ok] >= 0)


def test_pixel_mask_evaluates_only_the_sampled_pixels():
    scene = synth.random_scene(300, seed=56, deg=1, size=(0.05, 0.6))
    cam = synth.camera_identity(72, 56)
    full = O.render_solid(scene, cam)
    mask = (np.random.default_rng(4).uniform(size=(cam.H, cam.W)) < 0.2).astype(np.uint8)
    part = O.render_solid(scene, cam, pix_mask=mask)
    sel = mask.astype(bool)
    np.testing.assert_array_equal(part["id"][sel], full["id"][sel])
    np.testing.assert_array_equal(part["image"][:, sel], full["image"][:, sel])
    np.testing.assert_array_equal(part["flags"][sel], full["flags"][sel])
    assert (part["id"][~sel] == -1).all() and (part["flags"][~sel] == 0).all()


def test_ambiguous_cull_flags_only_the_triangles_own_pixels():
    """A triangle culled by a near-plane test within the FP32 band (one vertex a hair in
    front of the plane) marks the pixels of its bounding box, and no pixel far from it."""
    cam = synth.camera_identity(64, 48, fx=50.0)
    uv_c = np.array([[6.0, 6.0], [24.0, 8.0], [10.0, 22.0]])
    z_near = O.DEFAULT_CONSTS["z_near"]
    culled = one_tri_scene(cam, uv_c, np.array([z_near * (1 - 1e-7), 3.0, 3.0]))
    uv_o = np.array([[40.0, 26.0], [60.0, 30.0], [46.0, 44.0]])
    other = one_tri_scene(cam, uv_o, np.full(3, 3.0))
    ref = O.render_solid(stack(culled, other), cam)
    assert (ref["id"] != 0).all()                       # the first triangle is culled
    X, Y = np.meshgrid(np.arange(cam.W) + 0.5, np.arange(cam.H) + 0.5)

    def box(uv, pad):
        lo, hi = uv.min(0) - pad, uv.max(0) + pad
        return (X >= lo[0]) & (X <= hi[0]) & (Y >= lo[1]) & (Y <= hi[1])
    assert (ref["flags"][box(uv_c, 1)] != 0).all()
    # away from both triangles (the other one's edges carry band flags of their own)
    far = ~box(uv_c, 2) & ~box(uv_o, 2)
    assert far.sum() > 500 and (ref["flags"][far] == 0).all()
