"""Pins of the densification reference (Sec. 3.3: midpoint subdivision keeps the
combined area and region; small triangles are cloned with noise in their plane) and of
the size regulariser L_s = 2 / |(v1 - v0) x (v2 - v0)| (Sec. 3.4) with its gradient."""
import numpy as np

from oracle import densify as D


def _scene(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3, 3))
    sh = rng.standard_normal((n, 4, 3))
    return v, sh, rng.uniform(0.05, 0.95, n), rng.uniform(0.3, 3.0, n)


def _bary(p, tri):
    """Barycentric coordinates of points p [M,3] in the plane of tri [3,3]."""
    a, b, c = tri
    M = np.stack([b - a, c - a], 1)
    lam = np.linalg.lstsq(M, (p - a).T, rcond=None)[0].T
    return np.stack([1 - lam[:, 0] - lam[:, 1], lam[:, 0], lam[:, 1]], 1)


def test_subdivision_preserves_area_and_region():
    v, sh, o, s = _scene(20, 1)
    sel = np.array([3, 7, 11])
    nv, nsh, no, ns = D.subdivide(v, sh, o, s, sel, np.zeros((3, 2)), 0.1, tau_small=0.0)
    assert len(nv) == 20 + 9
    rng = np.random.default_rng(2)
    for k, i in enumerate(sel):
        kids = np.stack([nv[i]] + [nv[20 + 3 * k + j] for j in range(3)])
        np.testing.assert_allclose(D.area(kids).sum(), D.area(v[i:i + 1])[0], rtol=1e-12)
        np.testing.assert_allclose(D.area(kids), D.area(v[i:i + 1])[0] / 4, rtol=1e-12)
        # random points of the parent lie in exactly one child (up to the shared edges)
        w = rng.dirichlet([1, 1, 1], 500)
        pts = w @ v[i]
        inside = np.stack([np.all(_bary(pts, kid) >= -1e-12, axis=1) for kid in kids], 1)
        strict = np.stack([np.all(_bary(pts, kid) > 1e-9, axis=1) for kid in kids], 1)
        assert np.all(inside.sum(1) >= 1) and np.all(strict.sum(1) <= 1)
        # attributes copied
        for j in range(3):
            np.testing.assert_array_equal(nsh[20 + 3 * k + j], sh[i])
            assert no[20 + 3 * k + j] == o[i] and ns[20 + 3 * k + j] == s[i]
        assert no[i] == o[i]
    untouched = np.setdiff1d(np.arange(20), sel)
    np.testing.assert_array_equal(nv[untouched], v[untouched])


def test_small_triangles_are_cloned_in_plane():
    v, sh, o, s = _scene(10, 3)
    sel = np.array([2, 5])
    noise = np.array([[0.3, -1.2], [2.0, 0.5]])
    tau = 1e9                                        # every triangle counts as small
    nv, nsh, no, ns = D.subdivide(v, sh, o, s, sel, noise, 0.05, tau_small=tau)
    assert len(nv) == 12
    for k, i in enumerate(sel):
        clone = nv[10 + k]
        t = clone - v[i]
        np.testing.assert_allclose(t, np.broadcast_to(t[0], (3, 3)), atol=1e-15)   # a translation
        nrm = np.cross(v[i, 1] - v[i, 0], v[i, 2] - v[i, 0])
        assert abs(t[0] @ nrm) <= 1e-12 * np.linalg.norm(nrm)                         # in the plane
        np.testing.assert_allclose(np.linalg.norm(t[0]), 0.05 * np.hypot(*noise[k]), rtol=1e-12)
        # two overlapping copies composite to the original opacity
        np.testing.assert_allclose(1 - (1 - no[i]) * (1 - no[10 + k]), o[i], rtol=1e-12)
        np.testing.assert_array_equal(nv[i], v[i])


def test_size_regulariser_closed_form_and_finite_differences():
    tri = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]])   # |cross| = 1
    L, g = D.size_reg(tri)
    assert L == 2.0
    v, _, _, _ = _scene(6, 4)
    L, g = D.size_reg(v, weight=0.7)
    h = 1e-6
    for i in range(6):
        for a in range(3):
            for b in range(3):
                vp, vm = v.copy(), v.copy()
                vp[i, a, b] += h
                vm[i, a, b] -= h
                fd = (D.size_reg(vp, 0.7)[0] - D.size_reg(vm, 0.7)[0]) / (2 * h)
                np.testing.assert_allclose(g[i, a, b], fd, rtol=1e-5, atol=1e-7)
    # scale invariance: L_s of a triangle scaled by k is L_s / k^2
    np.testing.assert_allclose(D.size_reg(3.0 * v)[0], D.size_reg(v)[0] / 9.0, rtol=1e-12)
    # degenerate triangles contribute nothing
    deg = np.array([[[0.0, 0, 0], [1, 1, 1], [2, 2, 2]]])
    Ld, gd = D.size_reg(deg)
    assert Ld == 0.0 and np.all(gd == 0.0)
