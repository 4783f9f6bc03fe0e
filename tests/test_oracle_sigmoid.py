"""Pins of the oracle's sigmoid window (Eq. indicator2, I = sigmoid(-phi / sigma),
the variant the paper compares against): 1/2 on the boundary, above inside, below
outside, constant 1/2 as sigma grows, an indicator as sigma shrinks; the render, the
tight rectangle and the adjoint with this window."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth
from test_oracle_adjoint import _fd, _scene
from test_oracle_render import CAM, UV, one_tri_scene, pix_centres

SIG = dict(O.DEFAULT_CONSTS, window=O.WINDOW_SIGMOID)
SIG_EXACT = dict(O.EXACT_CONSTS, window=O.WINDOW_SIGMOID)


def test_boundary_inside_outside_and_limits():
    q = UV
    mids = (q + np.roll(q, -1, axis=0)) / 2                   # edge midpoints: phi = 0
    phi, I = O.window_sigmoid(q, 1.7, mids)
    np.testing.assert_allclose(phi, 0.0, atol=1e-12)
    np.testing.assert_allclose(I, 0.5, atol=1e-12)
    pts = pix_centres(CAM)
    ratio, _ = O.window(q, 1.0, pts)
    phi, I = O.window_sigmoid(q, 1.7, pts)
    r = O.tri2d(q)["r"]
    np.testing.assert_allclose(phi, -r * ratio, rtol=1e-12, atol=1e-12)   # phi(p) = ratio phi(s), phi(s) = -r
    assert np.all(I[ratio > 1e-9] > 0.5) and np.all(I[ratio < -1e-9] < 0.5)
    _, Ib = O.window_sigmoid(q, 1e9, pts)
    np.testing.assert_allclose(Ib, 0.5, atol=1e-7)             # globally supported as sigma grows
    _, Is = O.window_sigmoid(q, 1e-4, pts)
    far = np.abs(phi) > 0.05
    np.testing.assert_array_equal(np.round(Is[far]), (ratio[far] > 0).astype(float))


def test_single_triangle_render_is_the_window_blend():
    o, sigma = 0.8, 1.5
    rgb = np.array([0.2, 0.6, 0.9])
    cam = synth.camera_identity(48, 40, fx=40.0)
    cam.bg = np.array([0.05, 0.1, 0.0], np.float32)
    s = one_tri_scene(cam, UV, np.array([3.0, 4.0, 5.0]), rgb=rgb, o=o, sigma=sigma)
    ref = O.render(s, cam, SIG, brute=True)
    _, I = O.window_sigmoid(UV, sigma, pix_centres(cam))
    a = np.minimum(o * I, 0.99)
    a = np.where(o * I >= 1 / 255, a, 0.0).reshape(cam.H, cam.W)
    want = rgb[:, None, None] * a + cam.bg.astype(float)[:, None, None] * (1 - a)
    np.testing.assert_allclose(ref["image"], want, atol=1e-12)
    # the support exceeds the triangle: pixels outside it are lit
    ratio, _ = O.window(UV, 1.0, pix_centres(cam))
    assert np.any((ratio.reshape(cam.H, cam.W) < 0) & (a > 0))


def test_tight_rectangle_holds_the_support():
    rng = np.random.default_rng(61)
    for _ in range(5):
        o, sigma = rng.uniform(0.02, 0.95), rng.uniform(0.3, 3.0)
        s = one_tri_scene(CAM, UV, np.array([3.0, 4.0, 5.0]), o=o, sigma=sigma)
        info = O.tri_info(s, CAM, SIG)
        _, I = O.window_sigmoid(UV, sigma, pix_centres(CAM))
        lit = (o * I >= 1 / 255).reshape(CAM.H, CAM.W)
        if not lit.any():
            assert info["ntiles"][0] == 0
            continue
        x0, y0, x1, y1 = info["pix"][0]
        ys, xs = np.nonzero(lit)
        assert xs.min() >= x0 and xs.max() <= x1 and ys.min() >= y0 and ys.max() <= y1
        if o > 2 / 255:                                   # c < 0: dilated beyond the vertices
            assert info["f"][0] > 1.0


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_matches_central_differences(seed):
    scene = _scene(seed, n=4, deg=1, sigma=(0.8, 2.5))
    cam = synth.camera_identity(24, 24, fx=22.0)
    g = np.random.default_rng(200 + seed).standard_normal((3, 24, 24))
    ad = O.render_grad(scene, cam, g, SIG_EXACT)
    n = 4
    for key, shape in (("verts", (n, 3, 3)), ("opacity", (n,)), ("sigma", (n,))):
        fd = np.zeros(shape)
        for idx in np.ndindex(*shape):
            fd[idx] = _fd(scene, cam, g, SIG_EXACT, key, idx)[0]
        err = np.linalg.norm(ad[key] - fd) / np.linalg.norm(fd)
        assert err < 1e-6, (key, err)
