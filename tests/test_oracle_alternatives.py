"""Pins of the oracle's FP32 classifier and of the outcomes it lists for pixels whose
decisions FP32 cannot fix (Sec. 3.1: kept when alpha >= 1/255, front-to-back order by
triangle centre depth, the transmittance stop): each case puts one decision exactly
on its threshold and checks that both outcomes appear, each equal to its closed form;
the gradient flag is checked against an FP32 evaluation of the window."""
import numpy as np

import oracle as O
from paper_2505_19175_gb300 import synth
from test_oracle_render import UV, one_tri_scene, pix_centres, stack

CAM = synth.camera_identity(48, 40, fx=40.0)


def _alts_at(ref, cam, x, y):
    a = ref["alts"]
    return a[a["pix"] == y * cam.W + x]


def _has(alts, colour, T, nk, tol=1e-12):
    d = np.maximum(np.abs(alts["image"] - np.asarray(colour)[None]).max(1), np.abs(alts["T"] - T))
    return bool(np.any((d <= tol) & (alts["n_kept"] == nk)))


def _interior_pixel(cam, uv, sigma):
    """An interior pixel centre of the triangle and its window value."""
    ratio, I = O.window(uv, sigma, pix_centres(cam))
    k = int(np.argmin(np.abs(ratio - 0.5)))
    return k % cam.W, k // cam.W, float(I[k])


def test_alpha_at_the_skip_threshold_lists_both_outcomes():
    rgb = np.array([0.9, 0.3, 0.1])
    x, y, I = _interior_pixel(CAM, UV, 1.0)
    o = (1.0 / 255.0) / I * (1.0 + 1e-9)          # alpha = 1/255 to within FP32's band
    s = one_tri_scene(CAM, UV, np.full(3, 3.0), rgb=rgb, o=o, sigma=1.0)
    ref = O.render(s, CAM, flags=True)
    assert ref["flags"][y, x] & O.AMB_SKIP
    a = _alts_at(ref, CAM, x, y)
    al = o * I
    assert len(a) == 2
    assert _has(a, rgb * al, 1.0 - al, 1, tol=1e-9)        # kept: bg = 0
    assert _has(a, np.zeros(3), 1.0, 0)                     # skipped
    # away from the threshold the same scene flags nothing
    clean = O.render(one_tri_scene(CAM, UV, np.full(3, 3.0), rgb=rgb, o=0.5, sigma=1.0), CAM, flags=True)
    assert not (clean["flags"] & O.AMB_DECISION).any() and len(clean["alts"]) == 0


def test_transmittance_at_the_stop_threshold_lists_both_outcomes():
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    bg = np.array([0.3, 0.2, 0.1])
    cam = synth.camera_identity(48, 40, fx=40.0)
    cam.bg = bg.astype(np.float32)
    bgf = bg.astype(np.float32).astype(float)
    # two opaque layers (alpha clamped at 0.99): T after both is 1e-4, the stop threshold
    s = stack(one_tri_scene(cam, UV, np.full(3, 2.0), rgb=c1, o=1.0, sigma=1e-3),
              one_tri_scene(cam, UV, np.full(3, 3.0), rgb=c2, o=1.0, sigma=1e-3))
    ref = O.render(s, cam, flags=True)
    x, y, _ = _interior_pixel(cam, UV, 1e-3)
    assert ref["flags"][y, x] & O.AMB_STOP
    a = _alts_at(ref, cam, x, y)
    a1 = a2 = 0.99
    stopped = c1 * a1 + (1 - a1) * bgf
    went_on = c1 * a1 + c2 * a2 * (1 - a1) + (1 - a1) * (1 - a2) * bgf
    assert _has(a, stopped, 1 - a1, 1, tol=1e-12)
    assert _has(a, went_on, (1 - a1) * (1 - a2), 2, tol=1e-12)


def test_equal_depths_list_both_orders():
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    o1, o2 = 0.6, 0.5
    uv2 = UV[[1, 2, 0]] + np.array([1.5, -0.5])      # another triangle, same centroid depth
    s = stack(one_tri_scene(CAM, UV, np.full(3, 3.0), rgb=c1, o=o1, sigma=1e-3),
              one_tri_scene(CAM, uv2, np.array([2.5, 3.0, 3.5]), rgb=c2, o=o2, sigma=1e-3))
    info = O.tri_info(s, CAM)
    assert info["depth"][0] == info["depth"][1]
    ref = O.render(s, CAM, flags=True)
    r1, _ = O.window(UV, 1e-3, pix_centres(CAM))
    r2, _ = O.window(info["q"][1], 1e-3, pix_centres(CAM))
    both = np.nonzero((r1 > 0.3) & (r2 > 0.3))[0]
    assert len(both) > 10
    for k in both[:5]:
        x, y = k % CAM.W, k // CAM.W
        assert ref["flags"][y, x] & O.AMB_ORDER
        a = _alts_at(ref, CAM, x, y)
        a1 = o1 * r1[k] ** 1e-3
        a2 = o2 * r2[k] ** 1e-3
        T = (1 - a1) * (1 - a2)
        assert _has(a, c1 * a1 + c2 * a2 * (1 - a1), T, 2, tol=1e-9)   # id order
        assert _has(a, c2 * a2 + c1 * a1 * (1 - a2), T, 2, tol=1e-9)   # swapped


def test_listed_outcomes_contain_the_fp64_result():
    """On dense random scenes every listed pixel's outcomes include the image FP64
    computes (the walk that takes every decision as FP64 does), and no unflagged pixel
    lists any."""
    for seed, W, H in [(1, 100, 37), (4, 257, 129)]:
        scene = synth.random_scene(1500, seed=seed, deg=3, size=(0.05, 0.6), sigma=(0.3, 3.0))
        cam = synth.camera_identity(W, H)
        ref = O.render(scene, cam, flags=True)
        a = ref["alts"]
        assert len(a) > 0
        listed = np.unique(a["pix"])
        fl = ref["flags"].reshape(-1)
        assert np.all(fl[listed] & O.AMB_DECISION)
        assert not np.any(fl & O.AMB_UNRES)
        for p in listed:
            y, x = divmod(int(p), W)
            assert _has(a[a["pix"] == p], ref["image"][:, y, x], ref["T_final"][y, x], ref["n_kept"][y, x], tol=0.0)


def _fp32_window_slope(uv, sigma, pts):
    """sigma ratio^(sigma - 1) with the ratio evaluated as an FP32 renderer would: edge
    values m_i(p) = 1 - n_i . (p - s) / r, re-based on the FP32-rounded incenter s_hi
    (m_i = C_i + A_i (p.x - s_hi.x) + B_i (p.y - s_hi.y)), every coefficient and
    operation in FP32, ratio = min_i m_i."""
    t = O.tri2d(uv)
    s_hi = t["s"].astype(np.float32)
    s_lo = t["s"] - s_hi.astype(np.float64)
    dx = pts[:, 0].astype(np.float32) - s_hi[0]
    dy = pts[:, 1].astype(np.float32) - s_hi[1]
    ratio = np.full(len(pts), np.inf, np.float32)
    for i in range(3):
        a = -t["n"][i] / t["r"]
        A, B = np.float32(a[0]), np.float32(a[1])
        C = np.float32(1.0 - a[0] * s_lo[0] - a[1] * s_lo[1])
        ratio = np.minimum(ratio, C + A * dx + B * dy)
    r32 = ratio.astype(np.float64)
    return sigma * np.where(r32 > 0, r32, np.nan) ** (sigma - 1.0)


def test_gradient_flag_covers_the_fp32_window_slope():
    """Against an FP32 evaluation of the window's slope: where the oracle leaves a
    pixel's gradient unflagged, the FP32 slope is within the flag's 1e-4 of the FP64
    one; near the edges of a triangle with sigma < 1, far from the image origin, the
    FP32 slope is off by more and those pixels carry the flag."""
    cam = synth.camera_identity(640, 480, fx=300.0)
    uv = np.array([[503.3, 401.1], [541.2, 409.7], [515.4, 445.6]])
    sigma = 0.4
    s = one_tri_scene(cam, uv, np.full(3, 3.0), o=0.95, sigma=sigma)
    ref = O.render(s, cam, flags=True)
    pts = pix_centres(cam)
    ratio, I = O.window(uv, sigma, pts)
    kept = (ratio > 0) & (0.95 * I >= 1 / 255)
    slope64 = sigma * np.where(ratio > 0, ratio, np.nan) ** (sigma - 1.0)
    slope32 = _fp32_window_slope(uv, sigma, pts)
    rel = np.abs(slope32 / slope64 - 1.0)
    gflag = (ref["flags"].reshape(-1) & O.AMB_GRAD) != 0
    assert kept.sum() > 300
    assert np.nanmax(rel[kept & ~gflag]) <= 1e-4
    assert (kept & gflag).sum() > 0 and np.nanmax(rel[kept & gflag]) > 1e-4
    # the image itself is resolved at those pixels
    assert not np.any(ref["flags"].reshape(-1)[kept & gflag] & O.AMB_DECISION)


def test_gradient_flag_marks_a_tie_of_the_active_edge():
    """An isosceles triangle symmetric about the pixel-centre column x = 20.5: above the
    incenter the two slanted edges are equally near on that column, so which edge the
    gradient goes to is a tie FP32 may break either way."""
    uv = np.array([[8.5, 34.0], [32.5, 34.0], [20.5, 4.0]])
    s = one_tri_scene(CAM, uv, np.full(3, 3.0), o=0.8, sigma=1.0)
    ref = O.render(s, CAM, flags=True)
    t = O.tri2d(uv)
    g = (ref["flags"] & O.AMB_GRAD) != 0
    rows = [y for y in range(CAM.H) if 8 < y + 0.5 < t["s"][1] - 1.0]
    assert len(rows) > 5
    assert all(g[y, 20] for y in rows)
    assert not any(g[y, 18] or g[y, 23] for y in rows)
