"""Pins for the polynomial screens (Sec. 2.1, Eq. moment1d, Eq. oned)."""
import numpy as np
import pytest

from oracle import fe1d, screens


def test_q1_weights_are_cloud_in_cell():
    # q = 1: the two weights are the cloud-in-cell fractions divided by h
    h = 0.37
    d = np.linspace(-h / 2, h / 2, 11)
    w = screens.screen_weights_1d(1, h, d)
    assert np.allclose(w[:, 0] * h, 0.5 - d / h, atol=1e-15)
    assert np.allclose(w[:, 1] * h, 0.5 + d / h, atol=1e-15)


def test_q2_q3_closed_forms():
    # rational closed forms derived by hand from Eq. moment1d with equispaced nodes (t = delta/h)
    h = 1.0
    t = np.linspace(-0.5, 0.5, 7)
    w2 = screens.screen_weights_1d(2, h, t)
    ref2 = np.stack([0.75 * (20 * t ** 2 - 4 * t - 1), -0.75 * (20 * t ** 2 - 3), 0.75 * (20 * t ** 2 + 4 * t - 1)], 1)
    assert np.allclose(w2, ref2, atol=1e-13)
    Om3 = screens.moment_matrix_1d(3, 1.0)
    ref3 = np.array([[1 / 4, 3 / 8, 3 / 8, 1 / 4], [-1 / 8, -9 / 80, 9 / 80, 1 / 8],
                     [19 / 240, 3 / 160, 3 / 160, 19 / 240], [-9 / 160, -27 / 2240, 27 / 2240, 9 / 160]])
    assert np.allclose(Om3, ref3, atol=1e-15)
    w3 = screens.screen_weights_1d(3, h, t)
    ref = np.stack([-(280 * t ** 3 - 180 * t ** 2 - 30 * t + 9) / 24, (1400 * t ** 3 - 540 * t ** 2 - 630 * t + 171) / 108,
                    -(1400 * t ** 3 + 540 * t ** 2 - 630 * t - 171) / 108, (280 * t ** 3 + 180 * t ** 2 - 30 * t - 9) / 24], 1)
    assert np.allclose(w3, ref, atol=1e-12)


def patch_quadrature(h, ngl):
    """Tensor Gauss-Legendre on the 27-element patch [-3h/2, 3h/2]^3, element by element."""
    t, w = fe1d.gauss_legendre01(ngl)
    x = np.concatenate([(-1.5 + k + t) * h for k in range(3)])
    wx = np.concatenate([w * h] * 3)
    X, Y, Z = np.meshgrid(x, x, x, indexing='ij')
    W = wx[:, None, None] * wx[None, :, None] * wx[None, None, :]
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), W.ravel()


@pytest.mark.parametrize("q", [1, 2, 3])
def test_3d_screen_moments(q):
    # integral 1 and vanishing moments (x - delta)^l (y - delta)^m (z - delta)^n for l, m, n <= q,
    # not all zero (Eq. moments, Eq. momentmatrix), by direct 3-D quadrature of rho
    h = 0.5
    rng = np.random.default_rng(0)
    delta = rng.uniform(-h / 2, h / 2, 3)
    pts, W = patch_quadrature(h, q + 2)
    rho = screens.screen_density(q, h, delta, pts)
    rel = pts - delta
    for l in range(q + 1):
        for m in range(q + 1):
            for n in range(q + 1):
                mom = np.sum(W * rho * rel[:, 0] ** l * rel[:, 1] ** m * rel[:, 2] ** n)
                target = 1.0 if (l, m, n) == (0, 0, 0) else 0.0
                assert abs(mom - target) < 1e-11 * (h ** (l + m + n)) + 1e-12, (l, m, n, mom)


def test_q1_second_moment():
    # q = 1 leaves the second central moment 5 h^2 / 12 - delta^2 per axis (not cancelled)
    h = 1.0
    pts, W = patch_quadrature(h, 3)
    for d in (-0.4, 0.0, 0.3):
        delta = np.array([d, 0.1, -0.2])
        rho = screens.screen_density(1, h, delta, pts)
        m2 = np.sum(W * rho * (pts[:, 0] - d) ** 2)
        assert abs(m2 - (5 / 12 - d * d)) < 1e-13
    # and the screen is non-negative for q = 1 (cloud-in-cell), non-monotone for q = 2
    rho2 = screens.screen_density(2, h, np.array([0.3, 0.0, 0.0]), pts)
    assert screens.screen_density(1, h, np.array([0.3, 0.0, 0.0]), pts).min() >= -1e-15
    assert rho2.min() < 0
