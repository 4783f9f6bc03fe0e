"""Pins of the oracle's per-pixel sort (the per-pixel ordering the paper leaves to future
work after Supp. "Tile assignment"): each pixel's fragments composite in the order of
the depth of their triangle's plane along the pixel's ray, ties to the lower id.

The expected per-pixel depths come from perspective-correct interpolation (1/z is
affine in screen space, so 1/z(p) = sum_k lambda_k(p) / z_k with the screen-space
barycentrics lambda), not from the oracle's ray-plane intersection."""
import numpy as np

import oracle as O
from paper_2505_19175_gb300 import synth
from test_oracle_adjoint import _fd, _scene
from test_oracle_render import one_tri_scene, pix_centres, stack

PIXEL = dict(O.DEFAULT_CONSTS, sort=O.SORT_PIXEL)
EXACT_PIXEL = dict(O.EXACT_CONSTS, sort=O.SORT_PIXEL)


def _bary(uv, pts):
    a, b, c = uv
    M = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
    l12 = np.linalg.solve(M, (pts - a).T).T
    return np.stack([1 - l12[:, 0] - l12[:, 1], l12[:, 0], l12[:, 1]], 1)


def test_reduces_to_the_tile_sort_for_fronto_parallel_triangles():
    """Every triangle at one depth: per-pixel and centroid orders agree, so the two
    modes give the same image to the last bit."""
    rng = np.random.default_rng(3)
    cam = synth.camera_identity(64, 48, fx=50.0)
    parts = []
    for k in range(40):
        c = rng.uniform([4, 4], [60, 44])
        uv = c + rng.normal(0, 6, (3, 2))
        z = rng.uniform(2.0, 6.0)
        parts.append(one_tri_scene(cam, uv, np.full(3, z), rgb=rng.uniform(0, 1, 3), o=rng.uniform(0.2, 0.9),
                                   sigma=rng.uniform(0.5, 2.0)))
    s = stack(*parts)
    a = O.render(s, cam)
    b = O.render(s, cam, PIXEL)
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["n_kept"], b["n_kept"])


def test_crossing_triangles_composite_nearest_first():
    """A tilted triangle crossing a fronto-parallel one: on each side of the crossing
    line the nearer plane composites first (closed form in exact mode)."""
    cam = synth.camera_identity(64, 48, fx=50.0)
    uv_a = np.array([[4.0, 4.0], [60.0, 8.0], [20.0, 44.0]])
    uv_b = np.array([[58.0, 42.0], [6.0, 30.0], [50.0, 3.0]])
    za = np.array([2.0, 6.0, 5.0])                       # centroid 4.33: behind B per tile
    ca, cb = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.3, 0.8])
    oa, ob, sa, sb = 0.7, 0.6, 1.3, 0.8
    s = stack(one_tri_scene(cam, uv_a, za, rgb=ca, o=oa, sigma=sa),
              one_tri_scene(cam, uv_b, np.full(3, 4.0), rgb=cb, o=ob, sigma=sb))
    got = O.render(s, cam, EXACT_PIXEL)["image"]
    tile = O.render(s, cam, O.EXACT_CONSTS)["image"]
    pts = pix_centres(cam)
    _, Ia = O.window(uv_a, sa, pts)
    _, Ib = O.window(uv_b, sb, pts)
    al_a, al_b = oa * Ia, ob * Ib
    lam = _bary(uv_a, pts)
    z_a = 1.0 / (lam / za).sum(1)                        # perspective-correct depth of A
    a_front = z_a < 4.0
    both = (al_a > 0) & (al_b > 0)
    # away from the crossing line and from the triangles' edges
    ok = both & (np.abs(z_a - 4.0) > 1e-3) & (Ia > 1e-6) & (Ib > 1e-6)
    assert ok.sum() > 50 and (ok & a_front).sum() > 20 and (ok & ~a_front).sum() > 20
    front = np.where(a_front[:, None], ca * al_a[:, None], cb * al_b[:, None])
    back = np.where(a_front[:, None], cb * al_b[:, None], ca * al_a[:, None])
    f_al = np.where(a_front, al_a, al_b)
    want = front + back * (1.0 - f_al)[:, None] + 0.0   # background 0
    got_px = got.reshape(3, -1).T
    np.testing.assert_allclose(got_px[ok], want[ok], atol=1e-12)
    # the tile sort (centroid depths 4.33 and 4) puts B first everywhere: it differs
    # exactly where A is nearer
    tile_px = tile.reshape(3, -1).T
    diff = np.abs(tile_px - got_px).max(1) > 1e-9
    np.testing.assert_array_equal(diff[ok], a_front[ok])


def test_input_order_invariance():
    scene = synth.random_scene(300, seed=61, deg=1, size=(0.1, 0.6))
    cam = synth.camera_identity(80, 64)
    perm = np.random.default_rng(2).permutation(scene.n)
    s2 = synth.Scene(scene.verts[perm], scene.sh[perm], scene.opacity[perm], scene.sigma[perm], scene.sh_degree)
    a = O.render(scene, cam, PIXEL)["image"]
    b = O.render(s2, cam, PIXEL)["image"]
    np.testing.assert_array_equal(a, b)


def test_adjoint_matches_central_differences_per_pixel_sort():
    """The order is piecewise constant in the parameters: the adjoint through the
    per-pixel order matches FP64 central differences (tiny scene, exact mode)."""
    scene = _scene(11, n=6, deg=1)
    cam = synth.camera_identity(32, 32, fx=30.0)
    g = np.random.default_rng(11).standard_normal((3, 32, 32))
    ad = O.render_grad(scene, cam, g, EXACT_PIXEL)
    n = scene["verts"].shape[0]
    for key, shape in (("verts", (n, 3, 3)), ("opacity", (n,)), ("sigma", (n,))):
        fd = np.zeros(shape)
        for idx in np.ndindex(*shape):
            fd[idx] = _fd(scene, cam, g, EXACT_PIXEL, key, idx)[0]
        assert np.linalg.norm(fd) > 0
        err = np.linalg.norm(ad[key] - fd) / np.linalg.norm(fd)
        assert err < 1e-6, (key, err)
