"""Pins of the oracle's real spherical-harmonic basis (degree <= 3; Sec. 4: 48 colour
floats per triangle) against orthonormality and an independent library routine."""
import numpy as np
import pytest

import oracle as O


def _sphere_quadrature(n_theta=16, n_phi=32):
    """Gauss-Legendre in cos(theta) x uniform in phi: exact for polynomials of degree
    < 2 n_theta in z and trigonometric degree < n_phi in phi."""
    z, w = np.polynomial.legendre.leggauss(n_theta)
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    Z, PHI = np.meshgrid(z, phi, indexing="ij")
    Wt = np.repeat(w[:, None], n_phi, 1) * (2 * np.pi / n_phi)
    s = np.sqrt(1 - Z ** 2)
    d = np.stack([s * np.cos(PHI), s * np.sin(PHI), Z], -1).reshape(-1, 3)
    return d, Wt.reshape(-1)


def test_orthonormal_basis():
    d, w = _sphere_quadrature()
    Y = O.sh_eval(3, d)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_degree_zero_constant():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_eval(0, d)
    np.testing.assert_allclose(Y, 0.5 / np.sqrt(np.pi), rtol=1e-15)


def test_matches_scipy_complex_harmonics():
    """Real basis from scipy's complex Y_l^m (which carries the Condon-Shortley phase):
    m > 0: sqrt(2) (-1)^m Re Y_l^m; m < 0: sqrt(2) (-1)^m Im Y_l^|m|; m = 0: Y_l^0."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(1)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = O.sh_eval(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            c = sp.sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                ref = c.real
            elif m > 0:
                ref = np.sqrt(2) * (-1) ** m * c.real
            else:
                ref = np.sqrt(2) * (-1) ** m * c.imag
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12, err_msg=f"l={l} m={m}")
