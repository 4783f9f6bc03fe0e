"""Pins of the oracle's 2D geometry and window function against what the paper and
plane geometry fix (Sec. 3.1 "A new window function", Eq. indicator1; Supp.
"Depth-dependant scaling")."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "triangle_345.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        vals[k] = np.array([float(x) for x in v])
    return vals


def test_345_triangle_matches_hand_derivation():
    g = _golden()
    t = O.tri2d(g["q"])
    np.testing.assert_allclose(t["ell"], g["ell"], atol=1e-14)
    np.testing.assert_allclose(t["r"], g["r"][0], atol=1e-14)
    np.testing.assert_allclose(t["s"], g["s"], atol=1e-14)
    np.testing.assert_allclose(t["n"][0], g["n0"], atol=1e-14)
    np.testing.assert_allclose(t["n"][1], g["n1"], atol=1e-14)
    np.testing.assert_allclose(t["n"][2], g["n2"], atol=1e-14)
    np.testing.assert_allclose(t["d"], g["d"], atol=1e-14)
    ratio, I = O.window(g["q"], 2.0, g["p"])
    np.testing.assert_allclose(ratio[0], g["ratio"][0], atol=1e-14)
    np.testing.assert_allclose(I[0], g["I_sigma2"][0], atol=1e-14)


def test_orientation_does_not_flip_normals():
    q = np.array([[0, 0], [3, 0], [0, 4]], float)
    a = O.tri2d(q)
    b = O.tri2d(q[::-1])          # clockwise
    # same triangle: same incenter and inradius; normals still point outward
    np.testing.assert_allclose(a["s"], b["s"], atol=1e-14)
    np.testing.assert_allclose(a["r"], b["r"], atol=1e-14)
    for t, qq in ((a, q), (b, q[::-1])):
        c = qq.mean(0)
        for i in range(3):
            # centroid lies on the inner side of every edge
            assert t["n"][i] @ c + t["d"][i] < 0


def test_equilateral_inradius():
    a = 2.7
    q = np.array([[0, 0], [a, 0], [a / 2, a * np.sqrt(3) / 2]])
    t = O.tri2d(q)
    np.testing.assert_allclose(t["r"], a / (2 * np.sqrt(3)), rtol=1e-14)
    np.testing.assert_allclose(t["s"], q.mean(0), atol=1e-14)


def _rand_tris(seed, n=20):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        q = rng.uniform(-5, 5, (3, 2))
        e1, e2 = q[1] - q[0], q[2] - q[0]
        area = abs(e1[0] * e2[1] - e1[1] * e2[0])
        if area > 1.0:
            out.append(q)
    return out


def _bary(q, p):
    """Barycentric coordinates of points p [M,2] by a linear solve."""
    A = np.array([[q[0, 0], q[1, 0], q[2, 0]], [q[0, 1], q[1, 1], q[2, 1]], [1, 1, 1]])
    rhs = np.stack([p[:, 0], p[:, 1], np.ones(len(p))])
    return np.linalg.solve(A, rhs).T


def test_incenter_is_equidistant_and_window_is_one_there():
    for q in _rand_tris(1):
        t = O.tri2d(q)
        L = t["n"] @ t["s"] + t["d"]
        np.testing.assert_allclose(L, -t["r"], rtol=1e-12, atol=1e-12)
        ratio, I = O.window(q, 1.7, t["s"][None])
        np.testing.assert_allclose(ratio[0], 1.0, atol=1e-12)
        np.testing.assert_allclose(I[0], 1.0, atol=1e-12)


def test_incenter_is_argmin_of_phi_by_brute_force():
    """The paper defines s as the point where phi is minimal: search a fine grid."""
    for q in _rand_tris(2, 5):
        t = O.tri2d(q)
        lo, hi = q.min(0), q.max(0)
        xs = np.linspace(lo[0], hi[0], 801)
        ys = np.linspace(lo[1], hi[1], 801)
        X, Y = np.meshgrid(xs, ys)
        pts = np.stack([X.ravel(), Y.ravel()], 1)
        ratio, _ = O.window(q, 1.0, pts)
        k = np.argmax(ratio)                    # ratio = phi/phi(s): max where phi is min
        h = max(xs[1] - xs[0], ys[1] - ys[0])
        assert np.linalg.norm(pts[k] - t["s"]) < 4 * h
        assert ratio.max() <= 1.0 + 1e-12


def test_window_zero_on_edges_and_outside():
    rng = np.random.default_rng(3)
    for q in _rand_tris(4):
        # points on each edge
        w = rng.uniform(0, 1, 50)
        for i in range(3):
            a, b = q[(i + 1) % 3], q[(i + 2) % 3]
            pts = a[None] + w[:, None] * (b - a)[None]
            ratio, I = O.window(q, 0.8, pts)
            np.testing.assert_allclose(ratio, 0.0, atol=1e-12)
            assert np.all(I <= 1e-9)
        # random points outside
        pts = rng.uniform(-8, 8, (2000, 2))
        lam = _bary(q, pts)
        out = np.any(lam < -1e-9, axis=1)
        ratio, I = O.window(q, 0.8, pts[out])
        assert np.all(I[ratio < 0] == 0.0)
        assert np.all(ratio <= 1e-12)


def test_window_ratio_equals_normalised_barycentric_minimum():
    """phi(p)/phi(s) = min_i lambda_i(p) * perimeter / ell_i: an independent closed form
    (lambda from a linear solve; ell_i the side opposite vertex i)."""
    rng = np.random.default_rng(5)
    for q in _rand_tris(6):
        t = O.tri2d(q)
        pts = rng.uniform(-6, 6, (500, 2))
        lam = _bary(q, pts)
        P = t["ell"].sum()
        expect = np.min(lam * P / t["ell"][None, :], axis=1)
        ratio, _ = O.window(q, 1.0, pts)
        np.testing.assert_allclose(ratio, expect, rtol=1e-10, atol=1e-10)


def test_window_monotone_from_incenter_to_boundary():
    for q in _rand_tris(7, 5):
        t = O.tri2d(q)
        for v in q:
            w = np.linspace(0, 1, 200)
            pts = t["s"][None] + w[:, None] * (v - t["s"])[None]
            _, I = O.window(q, 1.3, pts)
            assert np.all(np.diff(I) <= 1e-15)
            np.testing.assert_allclose(I[0], 1.0, atol=1e-12)
            assert I[-1] <= 1e-12


def test_sigma_limits():
    """sigma -> 0 approaches the triangle's indicator; sigma -> inf a delta at s."""
    a = 4.0
    q = np.array([[0, 0], [a, 0], [a / 2, a * np.sqrt(3) / 2]])
    t = O.tri2d(q)
    rng = np.random.default_rng(8)
    pts = rng.uniform(-1, 5, (20000, 2))
    lam = _bary(q, pts)
    # distance to the nearest edge line
    dist = -(np.max(pts @ t["n"].T + t["d"][None], axis=1))
    inside = (dist >= 1e-2 * t["r"]) & np.all(lam > 0, axis=1)
    _, I = O.window(q, 1e-3, pts[inside])
    assert np.all(I > 0.99)
    far = np.linalg.norm(pts - t["s"][None], axis=1) >= 0.02 * t["r"]
    _, I = O.window(q, 1e3, pts[far])
    assert np.all(I < 1e-3)


@pytest.mark.parametrize("a", [0.5, 2.0, 7.3])
def test_scale_invariance(a):
    """Supp. "Depth-dependant scaling": I'(a p) = I(p) for the triangle scaled by a."""
    rng = np.random.default_rng(9)
    for q in _rand_tris(10, 5):
        pts = rng.uniform(-6, 6, (300, 2))
        _, I1 = O.window(q, 1.4, pts)
        _, I2 = O.window(a * q, 1.4, a * pts)
        np.testing.assert_allclose(I1, I2, rtol=1e-10, atol=1e-13)


def test_rigid_motion_invariance():
    rng = np.random.default_rng(11)
    th = 0.7
    Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    off = np.array([3.3, -1.2])
    for q in _rand_tris(12, 5):
        pts = rng.uniform(-6, 6, (300, 2))
        _, I1 = O.window(q, 0.9, pts)
        _, I2 = O.window(q @ Rm.T + off, 0.9, pts @ Rm.T + off)
        np.testing.assert_allclose(I1, I2, rtol=1e-9, atol=1e-12)
