"""Pins of the oracle's adjoint against FP64 central differences of its own forward
(the gradients the paper optimises, Sec. 3.3: vertices, sigma, opacity, SH)."""
import numpy as np
import pytest

import oracle as O
from paper_2505_19175_gb300 import synth


def _scene(seed, n=6, deg=3, sigma=(1.2, 2.5)):
    s = synth.random_scene(n, seed=seed, deg=deg, size=(0.25, 0.5), sigma=sigma, opacity=(0.3, 0.9),
                           sh_std=0.15, box=((-0.4, 0.4), (-0.3, 0.3), (2.5, 4.0)))
    return dict(verts=s.verts.astype(np.float64), sh=s.sh.astype(np.float64),
                opacity=s.opacity.astype(np.float64), sigma=s.sigma.astype(np.float64),
                sh_degree=deg)


def _loss(scene, cam, g, consts):
    return float(np.sum(O.render(scene, cam, consts, brute=True)["image"] * g))


def _fd(scene, cam, g, consts, key, idx, rel=1e-6):
    th = scene[key][idx]
    h = rel * max(1.0, abs(th))
    sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    sm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    sp[key][idx] = th + h
    sm[key][idx] = th - h
    return (_loss(sp, cam, g, consts) - _loss(sm, cam, g, consts)) / (2 * h), sp, sm


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_matches_central_differences_exact_mode(seed):
    scene = _scene(seed)
    cam = synth.camera_identity(32, 32, fx=30.0)
    g = np.random.default_rng(100 + seed).standard_normal((3, 32, 32))
    ad = O.render_grad(scene, cam, g, O.EXACT_CONSTS)
    n = scene["verts"].shape[0]
    for key, shape in (("verts", (n, 3, 3)), ("opacity", (n,)), ("sigma", (n,)), ("sh", scene["sh"].shape)):
        fd = np.zeros(shape)
        for idx in np.ndindex(*shape):
            fd[idx] = _fd(scene, cam, g, O.EXACT_CONSTS, key, idx)[0]
        a = ad[key]
        assert np.linalg.norm(fd) > 0
        err = np.linalg.norm(a - fd) / np.linalg.norm(fd)
        assert err < 1e-6, (key, err)
        np.testing.assert_allclose(a, fd, rtol=1e-5, atol=1e-7 * np.sqrt(np.mean(fd ** 2)) + 1e-12,
                                   err_msg=key)


def test_adjoint_soft_edges_small_sigma():
    """sigma < 1: the window has an infinite slope at the edges; away from them the
    adjoint still matches central differences."""
    scene = _scene(7, n=4, sigma=(0.4, 0.9))
    cam = synth.camera_identity(32, 32, fx=30.0)
    g = np.random.default_rng(7).standard_normal((3, 32, 32))
    ad = O.render_grad(scene, cam, g, O.EXACT_CONSTS)
    for key in ("opacity", "sigma"):
        fd = np.array([_fd(scene, cam, g, O.EXACT_CONSTS, key, (i,), rel=1e-7)[0] for i in range(4)])
        np.testing.assert_allclose(ad[key], fd, rtol=1e-5, atol=1e-9)


def test_adjoint_default_mode_where_no_decision_moves():
    """With the compositing thresholds on, compare only parameters whose +-h step changes
    no kept/skipped decision (the per-pixel kept counts are unchanged)."""
    scene = _scene(3, n=8, deg=1, sigma=(0.8, 2.0))
    scene["opacity"][:] = np.linspace(0.85, 0.98, 8)
    cam = synth.camera_identity(32, 32, fx=30.0)
    g = np.random.default_rng(3).standard_normal((3, 32, 32))
    ad = O.render_grad(scene, cam, g, O.DEFAULT_CONSTS)
    base = O.render(scene, cam, O.DEFAULT_CONSTS)["n_kept"]
    checked = 0
    for key in ("verts", "opacity", "sigma"):
        for idx in np.ndindex(*scene[key].shape):
            fd, sp, sm = _fd(scene, cam, g, O.DEFAULT_CONSTS, key, idx)
            if not (np.array_equal(O.render(sp, cam, O.DEFAULT_CONSTS)["n_kept"], base) and
                    np.array_equal(O.render(sm, cam, O.DEFAULT_CONSTS)["n_kept"], base)):
                continue
            checked += 1
            assert abs(ad[key][idx] - fd) <= 1e-5 * (abs(fd) + abs(ad[key][idx])) + 1e-8, (key, idx, ad[key][idx], fd)
    assert checked > 50


def test_masks_restrict_the_sum():
    """Gradients from a pixel subset equal those of the loss restricted to it; a
    triangle mask leaves other triangles at zero."""
    scene = _scene(4, n=5)
    cam = synth.camera_identity(32, 32, fx=30.0)
    g = np.random.default_rng(4).standard_normal((3, 32, 32))
    pm = np.zeros((32, 32), np.uint8)
    pm[8:20, 5:30] = 1
    a = O.render_grad(scene, cam, g * pm[None], O.EXACT_CONSTS)
    b = O.render_grad(scene, cam, g, O.EXACT_CONSTS, pix_mask=pm)
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14)
    tm = np.array([1, 0, 1, 0, 0], np.uint8)
    c = O.render_grad(scene, cam, g, O.EXACT_CONSTS, tri_mask=tm)
    full = O.render_grad(scene, cam, g, O.EXACT_CONSTS)
    for k in c:
        np.testing.assert_allclose(c[k][tm == 1], full[k][tm == 1], rtol=1e-12, atol=1e-14)
        assert np.all(c[k][tm == 0] == 0)
