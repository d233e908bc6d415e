"""Polynomial screens (oracle; test infrastructure).

Sec. 2.1: a charge in element tau gets a screen rho = sum_kappa c_kappa psi_kappa,
psi_kappa = omega_i(x) omega_j(y) omega_k(z) the global C0 order-q Lagrange
nodal functions of the (q+1)^3 nodes of the charge's element (Eq. oned), with
support on the 27-element patch [-3h/2, 3h/2]^3 around the element centre.
The separable form c_kappa = w^x_i w^y_j w^z_k, kappa = i + (q+1) j + (q+1)^2 k,
solves three (q+1)x(q+1) moment systems (Eq. moment1d):

    sum_i  bar-omega_i^(l) w_i = delta^l,   l = 0..q,
    bar-omega_i^(l) = int_{-3h/2}^{3h/2} x^l omega_i(x) dx   (Eq. cmomentsbasis).
"""
import numpy as np

from .fe1d import gauss_legendre01, lagrange_values


def omega_pieces(q, h, nodes=None):
    """Global C0 order-q nodal functions of the centre element's q+1 nodes.

    Returns, for node i, a list of (a, b, f) pieces: on [a, b], omega_i = f(x).
    The centre element is [-h/2, h/2]; its left vertex (i = 0) is also the right
    vertex of [-3h/2, -h/2], its right vertex (i = q) the left vertex of [h/2, 3h/2]."""
    out = []
    for i in range(q + 1):
        pieces = [(-0.5 * h, 0.5 * h, (lambda x, i=i: lagrange_values(q, (x + 0.5 * h) / h, nodes)[..., i]))]
        if i == 0:
            pieces.append((-1.5 * h, -0.5 * h, lambda x: lagrange_values(q, (x + 1.5 * h) / h, nodes)[..., q]))
        if i == q:
            pieces.append((0.5 * h, 1.5 * h, lambda x: lagrange_values(q, (x - 0.5 * h) / h, nodes)[..., 0]))
        out.append(pieces)
    return out


def moment_matrix_1d(q, h, nodes=None):
    """Omega[l, i] = bar-omega_i^(l), the centred 1-D moments (Eq. cmomentsbasis)."""
    t, w = gauss_legendre01(q + 2)
    Om = np.zeros((q + 1, q + 1))
    for i, pieces in enumerate(omega_pieces(q, h, nodes)):
        for (a, b, f) in pieces:
            x = a + (b - a) * t
            fx = f(x)
            for l in range(q + 1):
                Om[l, i] += (b - a) * np.sum(w * x ** l * fx)
    return Om


def screen_weights_1d(q, h, delta, nodes=None):
    """w_i(delta), i = 0..q, for offsets delta (any shape): solves Eq. moment1d.

    Output shape delta.shape + (q+1,), units 1/h."""
    delta = np.asarray(delta, dtype=np.float64)
    Om = moment_matrix_1d(q, h, nodes)
    rhs = np.stack([delta ** l for l in range(q + 1)], axis=-1)
    return np.linalg.solve(Om, rhs[..., None])[..., 0]


def screen_coefficients(q, h, delta3, nodes=None):
    """c_kappa(delta) = w^x_i w^y_j w^z_k with kappa = i + (q+1) j + (q+1)^2 k (Eq. oned).

    delta3: (..., 3) offsets from the element centre.  Returns (..., (q+1)^3), units 1/h^3."""
    delta3 = np.asarray(delta3, dtype=np.float64)
    wx = screen_weights_1d(q, h, delta3[..., 0], nodes)
    wy = screen_weights_1d(q, h, delta3[..., 1], nodes)
    wz = screen_weights_1d(q, h, delta3[..., 2], nodes)
    c = wz[..., :, None, None] * wy[..., None, :, None] * wx[..., None, None, :]
    return c.reshape(delta3.shape[:-1] + ((q + 1) ** 3,))


def screen_density(q, h, delta3, xs):
    """rho(x) of a unit charge at offset delta3 in the element centred at 0, at points xs (..., 3).

    Direct evaluation of sum_kappa c_kappa psi_kappa(x) (Eq. sumscreen) for moment checks."""
    c = screen_coefficients(q, h, np.asarray(delta3)[None, :])[0]
    xs = np.asarray(xs, dtype=np.float64)
    om = []
    pieces = omega_pieces(q, h)
    for a in range(3):
        vals = np.zeros(xs.shape[:-1] + (q + 1,))
        for i in range(q + 1):
            for (lo, hi, f) in pieces[i]:
                m = (xs[..., a] >= lo) & (xs[..., a] <= hi)
                v = np.where(m, f(np.clip(xs[..., a], lo, hi)), 0.0)
                # a shared vertex lies in two pieces; both give the same value there
                vals[..., i] = np.where(m, v, vals[..., i])
        om.append(vals)
    q1 = q + 1
    rho = np.zeros(xs.shape[:-1])
    for k in range(q1):
        for j in range(q1):
            for i in range(q1):
                rho += c[i + q1 * j + q1 * q1 * k] * om[0][..., i] * om[1][..., j] * om[2][..., k]
    return rho
