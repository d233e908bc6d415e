"""Pins for the load vector and the periodic FE mesh solve (Sec. 2.2, Eq. defineassign)."""
import itertools

import numpy as np
import pytest

from oracle import fe1d, fep3m, screens, tables


def element_stiffness_3d(p, h):
    """64 x 64 order-p hexahedral stiffness by direct 3-D quadrature of grad u_i . grad u_j."""
    t, w = fe1d.gauss_legendre01(p + 2)
    L = fe1d.lagrange_values(p, t)
    D = fe1d.lagrange_derivs(p, t) / h
    n1 = p + 1
    K = np.zeros((n1 ** 3, n1 ** 3))
    for gx, gy, gz in itertools.product(range(len(t)), repeat=3):
        wt = w[gx] * w[gy] * w[gz] * h ** 3
        grad = np.zeros((n1 ** 3, 3))
        for m in range(n1 ** 3):
            i, j, k = m % n1, (m // n1) % n1, m // n1 ** 2
            grad[m] = (D[gx, i] * L[gy, j] * L[gz, k], L[gx, i] * D[gy, j] * L[gz, k], L[gx, i] * L[gy, j] * D[gz, k])
        K += wt * grad @ grad.T
    return K


def test_kronecker_stiffness_equals_element_assembly():
    p, n, L = 3, 3, 1.0
    h = L / n
    Ke3 = element_stiffness_3d(p, h)
    N = p * n
    Kg = np.zeros((N ** 3, N ** 3))
    n1 = p + 1
    for ex, ey, ez in itertools.product(range(n), repeat=3):
        idx = []
        for m in range(n1 ** 3):
            i, j, k = m % n1, (m // n1) % n1, m // n1 ** 2
            idx.append((((p * ex + i) % N) * N + (p * ey + j) % N) * N + (p * ez + k) % N)
        idx = np.array(idx)
        Kg[np.ix_(idx, idx)] += Ke3
    ops = fep3m.MeshOperators(L, n)
    X = np.random.default_rng(0).normal(size=(N, N, N))
    assert np.abs(ops.apply_K(X).ravel() - Kg @ X.ravel()).max() < 1e-12


@pytest.mark.parametrize("n", [7, 9])
def test_solve_is_exact_and_mean_zero(n):
    ops = fep3m.MeshOperators(1.0, n)
    rng = np.random.default_rng(n)
    b = ops.neutralise(rng.normal(size=(3 * n,) * 3))
    phi = ops.solve(b)
    assert np.abs(ops.apply_K(phi) - b).max() < 1e-11 * np.abs(b).max()
    assert abs(np.sum(ops.w3() * phi)) < 1e-13


def manufactured_error(n):
    """Nodal max error of the FE solution of -Lap u = 4 pi rho, u = cos(2 pi x) cos(2 pi y) cos(2 pi z)."""
    L = 1.0
    ops = fep3m.MeshOperators(L, n)
    h = L / n
    t, w = fe1d.gauss_legendre01(10)
    lv = fe1d.lagrange_values(3, t)
    m1 = np.zeros(3 * n)
    for e in range(n):
        x = (e + t) * h
        for k in range(4):
            m1[(3 * e + k) % (3 * n)] += h * np.sum(w * np.cos(2 * np.pi * x) * lv[:, k])
    k2 = 3 * (2 * np.pi) ** 2
    b = k2 * m1[:, None, None] * m1[None, :, None] * m1[None, None, :]     # 4 pi int rho u_m
    phi = ops.solve(b)
    x = np.arange(3 * n) * h / 3
    u = np.cos(2 * np.pi * x)
    exact = u[:, None, None] * u[None, :, None] * u[None, None, :]
    return np.abs(phi - exact).max()


def test_manufactured_solution_converges_at_order_p_plus_1():
    e1, e2 = manufactured_error(8), manufactured_error(16)
    assert e2 < 2e-5
    assert e1 / e2 > 13.0, (e1, e2)          # h^4 for p = 3 (ratio -> 16)


def test_load_vector_matches_direct_quadrature():
    # one charge: b_m = 4 pi Q int rho u_m with rho evaluated directly (Eq. sumscreen)
    L, n = 1.0, 7
    h = L / n
    pos = np.array([[0.43, 0.51, 0.77]])
    Q = np.array([1.7])
    f = fep3m.forward(np.r_[pos, [[0.1, 0.1, 0.1]]], np.r_[Q, [0.0]], L, n, neutralise=False)
    b = f['b']
    bins = f['bins']
    e = bins['c3'][0]
    t, w = fe1d.gauss_legendre01(5)
    # integrate over the 27-element patch, element by element
    ref = {}
    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
        el = (e + np.array([dx, dy, dz])) % n
        lo = np.array([dx, dy, dz]) * h - h / 2             # relative to the charge's element centre
        X, Y, Z = np.meshgrid(lo[0] + t * h, lo[1] + t * h, lo[2] + t * h, indexing='ij')
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel() * h ** 3
        rho = screens.screen_density(1, h, bins['delta'][0], pts) * Q[0]
        lv = fe1d.lagrange_values(3, t)
        for m in range(64):
            i, j, k = m % 4, (m // 4) % 4, m // 16
            um = (lv[:, i][:, None, None] * lv[:, j][None, :, None] * lv[:, k][None, None, :]).ravel()
            key = tuple((3 * el + np.array([i, j, k])) % (3 * n))
            ref[key] = ref.get(key, 0.0) + 4 * np.pi * np.sum(W * rho * um)
    for key, val in ref.items():
        assert abs(b[key] - val) < 1e-13, (key, b[key], val)
    nz = np.argwhere(np.abs(b) > 1e-15)
    assert len(nz) == len(ref)
