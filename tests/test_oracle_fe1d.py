"""Pins for the 1-D finite elements of the mesh solve (Sec. 2.2)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fe1d


def exact_lagrange_matrices(p):
    """Exact rational element matrices on [0, 1] by integrating the Lagrange
    polynomials with Fraction arithmetic (independent of the float quadrature)."""
    nodes = [Fraction(k, p) for k in range(p + 1)]

    def poly(k):
        c = [Fraction(1)]
        for j, x in enumerate(nodes):
            if j == k:
                continue
            d = nodes[k] - x
            c = [(a if i < len(c) else 0) for i, a in enumerate(c + [0])]
            c = [(c[i - 1] if i > 0 else 0) / d - c[i] * x / d for i in range(len(c))]
        return c  # coefficients, ascending powers

    def mul(a, b):
        out = [Fraction(0)] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            for j, y in enumerate(b):
                out[i + j] += x * y
        return out

    def integ(a):
        return sum(c / (i + 1) for i, c in enumerate(a))

    def der(a):
        return [i * a[i] for i in range(1, len(a))] or [Fraction(0)]

    P = [poly(k) for k in range(p + 1)]
    M = [[integ(mul(P[i], P[j])) for j in range(p + 1)] for i in range(p + 1)]
    K = [[integ(mul(der(P[i]), der(P[j]))) for j in range(p + 1)] for i in range(p + 1)]
    I = [integ(P[i]) for i in range(p + 1)]
    return M, K, I


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_element_matrices_exact(p):
    Me, Ke = fe1d.element_matrices(p, 1.0)
    M, K, _ = exact_lagrange_matrices(p)
    assert np.allclose(Me, np.array(M, dtype=float), rtol=0, atol=1e-14)
    assert np.allclose(Ke, np.array(K, dtype=float), rtol=0, atol=1e-13)


def test_cubic_textbook_values():
    # equispaced cubic Lagrange element: mass h/1680 * [...], stiffness 1/(40 h) * [...]
    Me, Ke = fe1d.element_matrices(3, 2.0)
    M = np.array([[128, 99, -36, 19], [99, 648, -81, -36], [-36, -81, 648, 99], [19, -36, 99, 128]]) * 2.0 / 1680
    K = np.array([[148, -189, 54, -13], [-189, 432, -297, 54], [54, -297, 432, -189], [-13, 54, -189, 148]]) / (40 * 2.0)
    assert np.allclose(Me, M, atol=1e-14) and np.allclose(Ke, K, atol=1e-14)


def test_node_integrals_are_newton_cotes():
    # int of the cubic Lagrange functions = Simpson's 3/8 weights; a vertex is shared by 2 elements
    w = fe1d.node_integrals_periodic(3, 5, 0.2)
    assert np.allclose(w[0::3], 0.2 * 0.25) and np.allclose(w[1::3], 0.2 * 3 / 8) and np.allclose(w[2::3], 0.2 * 3 / 8)
    _, _, I = exact_lagrange_matrices(3)
    assert [float(x) for x in I] == [1 / 8, 3 / 8, 3 / 8, 1 / 8]


def test_periodic_matrix_identities():
    n, h = 6, 1.0 / 6
    M1, K1, Mpq = fe1d.periodic_matrices(3, n, h, 1)
    one = np.ones(3 * n)
    assert np.abs(K1 @ one).max() < 1e-12                       # stiffness kills constants
    assert np.allclose(M1 @ one, fe1d.node_integrals_periodic(3, n, h))
    assert np.allclose(M1, M1.T) and np.allclose(K1, K1.T)
    # columns of Mpq: int(hat_j * sum_i phi_i) = int hat_j = h
    assert np.allclose(Mpq.sum(axis=0), h)
    # the linear hats lie in the cubic space, so Mpq = M1 @ (cubic nodal values of the hats)
    x = np.arange(3 * n) / 3.0
    hats = np.maximum(0, 1 - np.abs(((x[:, None] - np.arange(n)[None, :]) + n / 2) % n - n / 2))
    assert np.allclose(Mpq, M1 @ hats, atol=1e-14)
