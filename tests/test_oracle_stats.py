"""Pins of the oracle's pruning statistics (Sec. 3.3 "Pruning": the largest blending
weight T o of a triangle over the pixels it is composited at, and the number of such
pixels, from which the two pruning rules are decided).

Each expected value is computed from the window function alone (``O.window``), not
from the compositing code it checks."""
import numpy as np

import oracle as O
from paper_2505_19175_gb300 import synth
from test_oracle_render import CAM, UV, one_tri_scene, pix_centres, stack

ALPHA_MIN = O.DEFAULT_CONSTS["alpha_min"]
ALPHA_MAX = O.DEFAULT_CONSTS["alpha_max"]


def _alpha(uv, o, sigma, cam=CAM):
    _, I = O.window(uv, sigma, pix_centres(cam))
    return np.minimum(o * I, ALPHA_MAX)


def test_single_triangle_counts_its_pixels_and_weighs_o():
    o, sigma = 0.7, 0.8
    s = one_tri_scene(CAM, UV, np.array([3.0, 3.5, 4.0]), o=o, sigma=sigma)
    st = O.render_stats(s, CAM)
    a = _alpha(UV, o, sigma)
    assert st["n_pix"][0] == int(np.sum(a >= ALPHA_MIN))
    assert st["max_weight"][0] == o          # nothing in front: T = 1
    assert st["amb"][0] == 0


def test_back_triangle_weight_is_attenuated_by_the_front_one():
    """Triangle B lies behind triangle F and inside it: B's weight at a pixel is
    (1 - alpha_F) o_B there, so its maximum is o_B (1 - min alpha_F over B's pixels)."""
    of, ob, sig = 0.6, 0.9, 0.5
    uv_b = (UV - UV.mean(0)) * 0.35 + UV.mean(0)
    front = one_tri_scene(CAM, UV, np.array([2.0, 2.0, 2.0]), o=of, sigma=sig)
    back = one_tri_scene(CAM, uv_b, np.array([5.0, 5.0, 5.0]), o=ob, sigma=sig)
    st = O.render_stats(stack(front, back), CAM)
    af = _alpha(UV, of, sig)
    ab = _alpha(uv_b, ob, sig)
    kf = af >= ALPHA_MIN
    kb = ab >= ALPHA_MIN
    T_b = np.where(kf, 1.0 - af, 1.0)
    assert st["n_pix"][1] == int(np.sum(kb))
    np.testing.assert_allclose(st["max_weight"][1], ob * T_b[kb].max(), rtol=1e-12)
    assert st["max_weight"][0] == of
    assert st["n_pix"][0] == int(np.sum(kf))


def test_counts_sum_to_the_composited_fragments_and_culled_triangles_are_zero():
    scene = synth.random_scene(300, seed=41, deg=1, size=(0.05, 0.5))
    cam = synth.camera_identity(80, 60)
    st = O.render_stats(scene, cam)
    ref = O.render(scene, cam)
    assert st["n_pix"].sum() == ref["n_kept"].sum()
    info = O.tri_info(scene, cam)
    culled = info["cull"] != 0
    assert np.all(st["n_pix"][culled] == 0) and np.all(st["max_weight"][culled] == 0)
    seen = st["n_pix"] > 0
    assert np.all(st["max_weight"][seen] <= np.asarray(scene.opacity, float)[seen] + 1e-15)
    assert np.all(st["max_weight"][seen] > 0)


def test_pruning_rules_on_views():
    """Two views: a triangle seen by both with more than one pixel survives the
    'twice with more than one pixel' rule; one seen by a single view does not."""
    # the second view is the left 32 columns of the first
    cams = [synth.camera_identity(48, 40, fx=40.0), synth.camera_identity(32, 40, fx=40.0, cx=24.0, cy=20.0)]
    z = np.array([3.0, 3.0, 3.0])
    both = one_tri_scene(cams[0], (UV - UV.mean(0)) * 0.3 + [22.0, 20.0], z, o=0.8)
    edge = one_tri_scene(cams[0], (UV - UV.mean(0)) * 0.15 + [40.0, 20.0], z * 1.5, o=0.8)
    scene = stack(both, edge)
    stats = [O.render_stats(scene, c) for c in cams]
    assert stats[0]["n_pix"][1] > 1 and stats[1]["n_pix"][1] == 0
    mw = np.stack([s["max_weight"] for s in stats])
    npix = np.stack([s["n_pix"] for s in stats])
    keep = O.prune_keep(mw, npix, tau_prune=0.1)
    assert keep.tolist() == [True, False]
    keep_lo = O.prune_keep(mw, npix, tau_prune=0.1, min_views=1)
    assert keep_lo.tolist() == [True, True]
    assert O.prune_keep(mw, npix, tau_prune=0.95).tolist() == [False, False]


def test_pruning_rule_thresholds_by_hand():
    """Each clause on a hand-made table: weights at, below and above tau; views with
    exactly one pixel do not count."""
    mw = np.array([[0.5, 0.49, 0.9, 0.9, 0.0],
                   [0.1, 0.30, 0.2, 0.9, 0.0]])
    npix = np.array([[2, 5, 1, 2, 0],
                     [2, 5, 7, 1, 0]])
    assert O.prune_keep(mw, npix, 0.5).tolist() == [True, False, False, False, False]
    assert O.prune_keep(mw, npix, 0.5, min_views=1).tolist() == [True, False, True, True, False]
    assert O.prune_keep(mw, npix, 0.5, min_pixels=1).tolist() == [True, False, True, True, False]
