"""Pins of the oracle's image against what the paper and the compositing rule fix
(Sec. 3.1: projection, window, front-to-back compositing by triangle centre depth;
Supp. "Tile assignment" for the tight rectangle)."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth

Y00 = 0.5 / np.sqrt(np.pi)     # textbook real SH Y_0^0


def backproject(cam, uv, z):
    """World points whose projection through ``cam`` is pixel position uv at depth z."""
    uv = np.asarray(uv, float)
    z = np.asarray(z, float)
    xc = np.stack([(uv[:, 0] - cam.cx) / cam.fx * z, (uv[:, 1] - cam.cy) / cam.fy * z, z], 1)
    R = np.asarray(cam.R, float)          # float32 rotation: use the true inverse
    return np.linalg.solve(R, (xc - np.asarray(cam.t, float)[None]).T).T


def one_tri_scene(cam, uv, z, rgb=(0.2, 0.6, 0.9), o=1.0, sigma=1.0, deg=0):
    v = backproject(cam, uv, z)[None]
    sh = np.zeros((1, (deg + 1) ** 2, 3))
    sh[0, 0] = (np.asarray(rgb) - 0.5) / Y00
    return dict(verts=v, sh=sh, opacity=np.array([o]), sigma=np.array([sigma]), sh_degree=deg)


def stack(*scenes):
    return dict(verts=np.concatenate([s["verts"] for s in scenes]),
                sh=np.concatenate([s["sh"] for s in scenes]),
                opacity=np.concatenate([s["opacity"] for s in scenes]),
                sigma=np.concatenate([s["sigma"] for s in scenes]),
                sh_degree=scenes[0]["sh_degree"])


def pix_centres(cam):
    X, Y = np.meshgrid(np.arange(cam.W) + 0.5, np.arange(cam.H) + 0.5)
    return np.stack([X.ravel(), Y.ravel()], 1)


CAM = synth.camera_identity(48, 40, fx=40.0)
UV = np.array([[6.3, 5.1], [41.2, 9.7], [15.4, 35.6]])


def test_projection_by_backprojection():
    cam = synth.camera_look_at((1.0, -0.5, -3.0), (0.2, 0.1, 0.5), 64, 48)
    s = one_tri_scene(cam, UV, np.array([3.0, 4.5, 2.2]))
    info = O.tri_info(s, cam)
    np.testing.assert_allclose(info["q"][0], UV, atol=1e-9)
    np.testing.assert_allclose(info["z"][0], [3.0, 4.5, 2.2], atol=1e-12)
    np.testing.assert_allclose(info["depth"][0], (3.0 + 4.5 + 2.2) / 3, atol=1e-12)


@pytest.mark.parametrize("exact", [True, False])
def test_single_opaque_triangle_returns_its_colour(exact):
    rgb = np.array([0.2, 0.6, 0.9])
    bg = np.array([0.05, 0.1, 0.0])
    cam = synth.camera_identity(48, 40, fx=40.0)
    cam.bg = bg.astype(np.float32)
    s = one_tri_scene(cam, UV, np.full(3, 3.0), rgb=rgb, o=1.0, sigma=1e-4)
    out = O.render(s, cam, O.EXACT_CONSTS if exact else O.DEFAULT_CONSTS)
    ratio, _ = O.window(UV, 1e-4, pix_centres(cam))
    ratio = ratio.reshape(cam.H, cam.W)
    img = out["image"]
    inside = ratio >= 0.05
    outside = ratio <= 0
    assert inside.sum() > 100 and outside.sum() > 100
    bgf = bg.astype(np.float32).astype(float)
    a = 1.0 if exact else 0.99
    for c in range(3):
        np.testing.assert_allclose(img[c][inside], a * rgb[c] + (1 - a) * bgf[c], atol=1e-3)
        np.testing.assert_array_equal(img[c][outside], bgf[c])


def test_two_layers_closed_form_and_order():
    cam = CAM
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    t1 = one_tri_scene(cam, UV, np.full(3, 2.0), rgb=c1, o=0.7, sigma=1.0)
    uv2 = UV + np.array([3.0, 2.0])
    t2 = one_tri_scene(cam, uv2, np.full(3, 4.0), rgb=c2, o=0.6, sigma=1.0)
    P = pix_centres(cam)
    r1, _ = O.window(UV, 1.0, P)
    r2, _ = O.window(uv2, 1.0, P)
    a1 = 0.7 * np.maximum(r1, 0)
    a2 = 0.6 * np.maximum(r2, 0)
    for scene, near_first in ((stack(t1, t2), True), (stack(t2, t1), True)):
        out = O.render(scene, cam, O.EXACT_CONSTS)
        for c in range(3):
            exp = c1[c] * a1 + c2[c] * a2 * (1 - a1)
            np.testing.assert_allclose(out["image"][c].ravel(), exp, atol=1e-12)
        np.testing.assert_allclose(out["T_final"].ravel(), (1 - a1) * (1 - a2), atol=1e-12)
    # move the second triangle in front: the order flips
    t2n = one_tri_scene(cam, uv2, np.full(3, 1.5), rgb=c2, o=0.6, sigma=1.0)
    out = O.render(stack(t1, t2n), cam, O.EXACT_CONSTS)
    for c in range(3):
        exp = c2[c] * a2 + c1[c] * a1 * (1 - a2)
        np.testing.assert_allclose(out["image"][c].ravel(), exp, atol=1e-12)


def test_skip_below_alpha_min_and_clamp():
    cam = CAM
    P = pix_centres(cam)
    t = one_tri_scene(cam, UV, np.full(3, 3.0), rgb=(1, 1, 1), o=0.995, sigma=0.7)
    r, _ = O.window(UV, 0.7, P)
    a = 0.995 * np.maximum(r, 0) ** 0.7
    out = O.render(t, cam, O.DEFAULT_CONSTS)
    exp = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)
    np.testing.assert_allclose(out["image"][0].ravel(), exp, atol=1e-12)
    np.testing.assert_array_equal(out["n_kept"].ravel(), (a >= 1 / 255).astype(int))


def test_transmittance_stop_rule():
    cam = CAM
    layers = [one_tri_scene(cam, UV, np.full(3, 2.0 + 0.1 * k), rgb=(0.5, 0.5, 0.5), o=0.8, sigma=1e-3)
              for k in range(8)]
    out = O.render(stack(*layers), cam, O.DEFAULT_CONSTS)
    r, I = O.window(UV, 1e-3, pix_centres(cam))
    inside = (r >= 0.05).reshape(cam.H, cam.W)
    # all layers share the footprint: T after k layers = (1 - 0.8 I)^k ~ 0.2^k, so
    # 5 layers stay above 1e-4 and a sixth would take T below it
    a = 0.8 * I.reshape(cam.H, cam.W)[inside]
    assert np.all((1 - a) ** 6 < 1e-4) and np.all((1 - a) ** 5 >= 1e-4)
    assert np.all(out["n_kept"][inside] == 5)
    np.testing.assert_allclose(out["T_final"][inside], (1 - a) ** 5, rtol=1e-12)


def test_near_plane_and_degenerate_cull():
    cam = CAM
    s = one_tri_scene(cam, UV, np.array([3.0, 0.1, 3.0]), o=0.9)
    out = O.render(s, cam)
    assert np.all(out["image"] == 0) and np.all(out["T_final"] == 1)
    assert O.tri_info(s, cam)["cull"][0] == 1
    flat = one_tri_scene(cam, np.array([[5.0, 5.0], [20.0, 5.0], [35.0, 5.0 + 1e-7]]), np.full(3, 3.0))
    assert O.tri_info(flat, cam)["cull"][0] == 2


def test_order_invariance_under_permutation():
    s = synth.random_scene(60, seed=3, deg=3)
    cam = synth.camera_identity(64, 48)
    a = O.render(s, cam)
    perm = np.random.default_rng(4).permutation(s.n)
    b = O.render(s.permuted(perm), cam)
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["T_final"], b["T_final"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fast_mode_bit_identical_to_brute_force(seed):
    s = synth.random_scene(150, seed=seed, deg=2)
    cam = synth.camera_identity(72, 56)
    a = O.render(s, cam, brute=True, flags=True)
    b = O.render(s, cam, brute=False, flags=True)
    for k in ("image", "T_final", "n_kept", "flags", "err"):
        np.testing.assert_array_equal(a[k], b[k])


def test_rigid_world_motion_with_compensating_camera():
    s = synth.random_scene(80, seed=5, deg=0)
    cam = synth.camera_look_at((0.3, -0.2, -0.5), (0.0, 0.0, 3.0), 64, 48)
    th = 0.9
    Q = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    Q = Q @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    a = np.array([1.5, -2.0, 0.7])
    v2 = s.verts.astype(float) @ Q.T + a
    R2 = cam.R.astype(float) @ Q.T
    t2 = cam.t.astype(float) - R2 @ a
    cam2 = dict(R=R2, t=t2, fx=cam.fx, fy=cam.fy, cx=cam.cx, cy=cam.cy, W=cam.W, H=cam.H, bg=cam.bg)
    s2 = dict(verts=v2, sh=s.sh, opacity=s.opacity, sigma=s.sigma, sh_degree=0)
    i1 = O.render(s, cam)["image"]
    i2 = O.render(s2, cam2)["image"]
    np.testing.assert_allclose(i1, i2, atol=1e-9)


def test_view_dependent_colour_degree_one():
    """Only c_{1,+1} (the x-linear basis function, index l^2 + l + m = 3) set: colour
    = 0.5 + sqrt(3/(4 pi)) dir_x c, dir from the camera centre to the centroid."""
    cam = synth.camera_look_at((2.0, -1.0, -1.0), (0.0, 0.0, 3.0), 64, 48)
    v = backproject(cam, UV, np.full(3, 4.0))[None]
    sh = np.zeros((1, 4, 3))
    sh[0, 3] = [0.3, -0.2, 0.1]
    s = dict(verts=v, sh=sh, opacity=np.array([0.5]), sigma=np.array([1.0]), sh_degree=1)
    info = O.tri_info(s, cam)
    d = v[0].mean(0) - cam.position()
    d /= np.linalg.norm(d)
    np.testing.assert_allclose(info["dir"][0], d, atol=1e-12)
    np.testing.assert_allclose(info["rgb"][0], np.maximum(0, 0.5 + np.sqrt(3 / (4 * np.pi)) * d[0] * sh[0, 3]),
                               atol=1e-12)


def test_tight_rectangle():
    """Supp. "Tile assignment": every pixel with o I >= tau lies in the rectangle; the
    shrunk triangle's vertices lie on the o I = tau level set; the rectangle is inside
    the vertex box and shrinks as sigma grows or o falls."""
    tau = O.DEFAULT_CONSTS["alpha_min"]
    cam = synth.camera_identity(96, 80, fx=80.0)
    P = pix_centres(cam)
    rng = np.random.default_rng(6)
    for trial in range(20):
        uv = rng.uniform([5, 5], [90, 75], (3, 2))
        o = rng.uniform(0.05, 1.0)
        sig = np.exp(rng.uniform(np.log(0.2), np.log(4.0)))
        s = one_tri_scene(cam, uv, np.full(3, 3.0), o=o, sigma=sig)
        info = O.tri_info(s, cam)
        if info["cull"][0] != 0:
            continue
        r, I = O.window(uv, sig, P)
        hit = (o * I >= tau).reshape(cam.H, cam.W)
        x0, y0, x1, y1 = info["pix"][0]
        ys, xs = np.nonzero(hit)
        if info["rect_state"][0] == 0:
            assert np.all((xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1))
            q = info["q"][0]
            rect = info["rect"][0]
            assert rect[0] >= q[:, 0].min() - 1e-9 and rect[2] <= q[:, 0].max() + 1e-9
            assert rect[1] >= q[:, 1].min() - 1e-9 and rect[3] <= q[:, 1].max() + 1e-9
            # shrunk vertices sit on the cutoff level set
            sc = info["s"][0]
            f = info["f"][0]
            w = sc[None] + f * (q - sc[None])
            rw, Iw = O.window(q, sig, w)
            # in ratio space (well conditioned even when the cutoff ratio is tiny)
            np.testing.assert_allclose(rw, (tau / o) ** (1 / sig), rtol=1e-6, atol=1e-12)
            # monotone shrinking
            prev = rect
            for sig2 in (sig * 1.5, sig * 3.0):
                r2 = O.tri_info(one_tri_scene(cam, uv, np.full(3, 3.0), o=o, sigma=sig2), cam)["rect"][0]
                assert r2[0] >= prev[0] - 1e-12 and r2[2] <= prev[2] + 1e-12
                assert r2[1] >= prev[1] - 1e-12 and r2[3] <= prev[3] + 1e-12
                prev = r2
            r3 = O.tri_info(one_tri_scene(cam, uv, np.full(3, 3.0), o=o * 0.5, sigma=sig), cam)
            if r3["rect_state"][0] == 0:
                r3 = r3["rect"][0]
                assert r3[0] >= rect[0] - 1e-12 and r3[2] <= rect[2] + 1e-12
        else:
            assert hit.sum() == 0


def test_tile_pairs_cover_every_contributing_tile():
    s = synth.random_scene(200, seed=7, deg=1)
    cam = synth.camera_identity(80, 64)
    tiles, ids = O.tile_pairs(s, cam)
    out = O.render(s, cam)
    info = O.tri_info(s, cam)
    tx = (cam.W + 15) // 16
    have = set(zip(tiles.tolist(), ids.tolist()))
    P = pix_centres(cam)
    for t in range(s.n):
        if info["cull"][t]:
            continue
        q = info["q"][t]
        _, I = O.window(q.reshape(-1), float(s.sigma[t]), P)
        hit = np.nonzero(float(s.opacity[t]) * I >= 1 / 255)[0]
        for p in hit:
            x, y = p % cam.W, p // cam.W
            assert ((y // 16) * tx + x // 16, t) in have
    # ordered by tile, then depth, then id
    d = info["depth"][ids]
    key_ok = (np.diff(tiles) > 0) | ((np.diff(tiles) == 0) & ((np.diff(d) > 0) | ((np.diff(d) == 0) & (np.diff(ids) > 0))))
    assert np.all(key_ok)
    assert out["image"].shape == (3, cam.H, cam.W)
