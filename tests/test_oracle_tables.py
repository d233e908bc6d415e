"""Pins for the basis-screen potential table (Eq. screenintegral, Eq. sc, Remark of Sec. 4)."""
import itertools

import numpy as np
import pytest

from oracle import fe1d, screens, tables


def cube_potential_closed_form(x, lo, hi):
    """Potential int dxi / |x - xi| of a uniform unit-density box, closed form
    (inclusion-exclusion over the corners of the antiderivative of 1/r)."""
    def F(u, v, w):
        r = np.sqrt(u * u + v * v + w * w)
        return (v * w * np.log(u + r) + u * w * np.log(v + r) + u * v * np.log(w + r)
                - 0.5 * u * u * np.arctan(v * w / (u * r)) - 0.5 * v * v * np.arctan(u * w / (v * r))
                - 0.5 * w * w * np.arctan(u * v / (w * r)))
    tot = 0.0
    for a, b, c in itertools.product((0, 1), repeat=3):
        u = (hi[0] if a else lo[0]) - x[0]
        v = (hi[1] if b else lo[1]) - x[1]
        w = (hi[2] if c else lo[2]) - x[2]
        tot += (-1) ** (3 - a - b - c) * F(u, v, w)
    return tot


def test_far_field_quadrature_matches_closed_form():
    lo, hi = np.array([-1.0, -0.5, 0.0]), np.array([0.0, 1.0, 1.0])
    qp, qw = tables.box_quadrature(lo, hi, 8)
    for x in ([6.3, 1.7, -2.9], [-7.1, 7.9, 0.4], [8.0, -8.0, 8.0]):
        x = np.array(x)
        ref = cube_potential_closed_form(x, lo, hi)
        val = tables.coulomb_quadrature(x[None, :], qp, qw)[0]
        assert abs(val - ref) < 1e-12 * abs(ref), (val, ref)   # the closed form itself cancels ~3 digits


def test_hat_far_field_has_no_quadrupole():
    # the hat has unit mass, zero dipole and isotropic second moments (1/6 per axis), so its
    # potential is 1/R + O(R^-5); its fourth moments give the R^-5 term
    rng = np.random.default_rng(3)
    for _ in range(5):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        R = 7.0
        x = R * u
        val = tables.hat_potential_continuum(x[None, :])[0]
        # hexadecapole term of a cubic-symmetric density: moments m4 = int x^4 psi = 1/15,
        # m22 = int x^2 y^2 psi = 1/36; Phi_4 = (35/8)(m4 - 3 m22)(sum u^4 - 3/5) / R^5
        m4, m22 = 1 / 15, 1 / 36
        phi4 = 35 / 8 * (m4 - 3 * m22) * (np.sum(u ** 4) - 0.6) / R ** 5
        assert abs(val - 1 / R - phi4) < 2e-7, (val - 1 / R, phi4)


@pytest.fixture(scope="module")
def table():
    return tables.basis_screen_table()


def test_table_cubic_symmetry(table):
    H, _ = table
    for perm in itertools.permutations(range(3)):
        assert np.abs(H - H.transpose(perm)).max() < 1e-13
    for ax in range(3):
        assert np.abs(H - np.flip(H, axis=ax)).max() < 1e-13


def test_table_solves_dirichlet_problem(table):
    # interior rows of the Galerkin system hold: K H = 4 pi Mpq psi at every interior node
    H, x1 = table
    p, n = 3, 16
    Me, Ke, Mpq_e = fe1d.element_matrices(p, 1.0, 1)
    M1 = fe1d.assemble_open(Me, n, p)
    K1 = fe1d.assemble_open(Ke, n, p)
    # independent right-hand side: int hat * phi_k by quadrature of the product on each element
    t, w = fe1d.gauss_legendre01(6)
    m1 = np.zeros(p * n + 1)
    for e in range(n):
        x = -8 + e + t
        hat = np.maximum(0.0, 1 - np.abs(x))
        m1[p * e:p * e + p + 1] += np.einsum('g,g,gk->k', w, hat, fe1d.lagrange_values(p, t))
    rhs = 4 * np.pi * m1[:, None, None] * m1[None, :, None] * m1[None, None, :]
    res = tables.stiffness_apply(K1, M1, H) - rhs
    assert np.abs(res[1:-1, 1:-1, 1:-1]).max() < 1e-13
    # boundary rows carry the continuum potential
    pts = np.array([[x1[0], x1[5], x1[40]], [x1[-1], x1[-1], x1[20]]])
    assert np.allclose([H[0, 5, 40], H[-1, -1, 20]], tables.hat_potential_continuum(pts), atol=1e-15)


def test_table_close_to_continuum(table):
    # the FE solution differs from the continuum potential only by discretisation error
    H, x1 = table
    c = 24
    for r in range(1, 5):
        for node in ((c + 3 * r, c, c), (c + 3 * r, c + 3 * r, c), (c + r, c + 2 * r, c - r)):
            x = np.array([x1[i] for i in node])
            cont = tables.hat_potential_continuum(x[None, :], ngl=24)[0]
            assert abs(H[node] - cont) < 3e-3 / r ** 2, (node, H[node], cont)


def test_table_box_size_converged():
    # boundary values from the continuum potential make the kept part insensitive to the box
    a = tables.kept_table(half_width=8)
    b = tables.kept_table(half_width=6)
    assert np.abs(a - b).max() < 2e-6


def test_screened_potential_decays_like_r_minus_3():
    # Sec. 2.1 / Fig. decayavg: for q = 1 the charge-plus-screen potential decays like R^-(q+2)
    h = 1.0
    delta = np.array([0.23, -0.11, 0.37])
    c = screens.screen_coefficients(1, h, delta[None, :])[0] * h ** 3
    rng = np.random.default_rng(1)
    dirs = rng.normal(size=(16, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    vals = {}
    for R in (4.0, 8.0):
        x = delta + R * dirs
        phi_sc = np.zeros(len(x))
        for kap in range(8):
            v = np.array([kap & 1, (kap >> 1) & 1, (kap >> 2) & 1]) - 0.5
            phi_sc += c[kap] * tables.hat_potential_continuum(x - v, ngl=12)
        vals[R] = np.sqrt(np.mean((1.0 / R - phi_sc) ** 2))
    slope = np.log(vals[8.0] / vals[4.0]) / np.log(2.0)
    assert -3.3 < slope < -2.7, slope
