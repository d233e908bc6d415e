"""Basis-screen potential table for q = 1 (oracle; test infrastructure).

Sec. 2.4 evaluates the screen potential (Eq. screenintegral) through tables of
basis-function potentials (Eq. sc).  The Remark of Sec. 4 says how the tables
used in the experiments were made: for each basis screen, a Dirichlet FE
solution of Poisson's equation in a domain larger than the part kept, with the
order-p FE, stored as order-p nodal values so that it is evaluated exactly like
the mesh potential.

For q = 1 the basis screen of a vertex is the trilinear hat psi_v (height 1,
support the 8 elements around the vertex); every vertex hat is a translate of
the same one, so one table serves all of them.  Readings fixed here (the paper
leaves them open):
  * units: -Laplace(H) = 4*pi*psi, so that a point charge Q has potential Q/R
    (Eq. potential); mesh size h = 1 (at size h the potential is h^2 H(x/h));
  * domain: the cube [-B, B]^3 (B = half_width elements) centred on the vertex,
    meshed by the same uniform elements as the global mesh (node-aligned);
  * boundary values: the continuum potential int psi(xi)/|x - xi| dxi of the hat
    at the boundary nodes (Eq. screenintegral), by tensor Gauss-Legendre
    quadrature on the hat's 8 polynomial pieces;
  * kept part: the nodal values on the 8^3 elements around the vertex, i.e.
    positions -4 .. 4 in steps of 1/p (what a 7^3-element short-range block
    needs for any of the 8 vertices of any of its source elements).
"""
import functools

import numpy as np
import scipy.linalg

from .fe1d import assemble_open, element_matrices, gauss_legendre01, lagrange_values


def hat_quadrature(ngl=8):
    """Points and weights*density for int psi(xi) f(xi) dxi, psi = prod(1-|xi_a|) on [-1,1]^3."""
    t, w = gauss_legendre01(ngl)
    xs, ws = [], []
    for lo in (-1.0, 0.0):
        x = lo + t
        xs.append(x)
        ws.append(w * (1.0 - np.abs(x)))
    x1 = np.concatenate(xs)
    w1 = np.concatenate(ws)
    X, Y, Z = np.meshgrid(x1, x1, x1, indexing='ij')
    W = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel()


def box_quadrature(lo, hi, ngl=8):
    """Tensor Gauss-Legendre points/weights of a uniform unit-density box [lo, hi] (3-vectors)."""
    t, w = gauss_legendre01(ngl)
    pts = [lo[a] + (hi[a] - lo[a]) * t for a in range(3)]
    wts = [(hi[a] - lo[a]) * w for a in range(3)]
    X, Y, Z = np.meshgrid(*pts, indexing='ij')
    W = wts[0][:, None, None] * wts[1][None, :, None] * wts[2][None, None, :]
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel()


def coulomb_quadrature(points, qpts, qwts, chunk=2048):
    """sum_g qwts_g / |x - qpts_g| for each x in points (x well away from qpts)."""
    points = np.asarray(points, dtype=np.float64)
    out = np.empty(len(points))
    for s in range(0, len(points), chunk):
        d = points[s:s + chunk, None, :] - qpts[None, :, :]
        out[s:s + chunk] = (qwts[None, :] / np.sqrt(np.einsum('pgk,pgk->pg', d, d))).sum(axis=1)
    return out


def hat_potential_continuum(points, ngl=8):
    """Continuum potential of the unit hat, int psi(xi)/|x-xi| dxi (Eq. screenintegral), h = 1."""
    qp, qw = hat_quadrature(ngl)
    return coulomb_quadrature(points, qp, qw)


def kron_apply(A, B, C, X):
    """(A (x) B (x) C) X on an array indexed [ix, iy, iz]: A acts on x, B on y, C on z.

    Each factor is one matrix product over its axis (tensordot, i.e. BLAS)."""
    Y = np.tensordot(A, X, axes=(1, 0))                          # [a, j, k]
    Y = np.moveaxis(np.tensordot(B, Y, axes=(1, 1)), 0, 1)       # [a, b, k]
    return np.tensordot(Y, C, axes=(2, 1))                       # [a, b, c]


def stiffness_apply(K1, M1, X):
    """K X with K = K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1 (Sec. 2.2, tensor-product mesh)."""
    return kron_apply(K1, M1, M1, X) + kron_apply(M1, K1, M1, X) + kron_apply(M1, M1, K1, X)


@functools.lru_cache(maxsize=4)
def basis_screen_table(p=3, half_width=8, ngl=8):
    """FE potential H of the unit vertex hat on the box [-B, B]^3 (h = 1), all nodes.

    Returns (H, x1): H[ix, iy, iz] at node positions x1[ix], x1[iy], x1[iz],
    x1 = -B + k/p, k = 0..2*B*p.  Galerkin: K_II H_I = 4*pi*(M_pq psi)_I - K_IB H_B,
    solved exactly by fast diagonalisation (Lynch-Rice-Thomas) of the 1-D
    Dirichlet pencils (K1_II, M1_II)."""
    n = 2 * half_width
    x1 = -half_width + np.arange(p * n + 1) / p
    Me, Ke, Mpq_e = element_matrices(p, 1.0, 1)
    M1 = assemble_open(Me, n, p)
    K1 = assemble_open(Ke, n, p)
    # 1-D mixed-mass column of the hat at the centre vertex: int phi^p_k(x) hat(x) dx
    c = half_width          # the centre vertex is the left end of element c
    m1 = np.zeros(p * n + 1)
    m1[p * (c - 1):p * c + 1] += Mpq_e[:, 1]     # element left of the vertex: hat rises (Q1 node 1)
    m1[p * c:p * (c + 1) + 1] += Mpq_e[:, 0]     # element right of the vertex: hat falls (Q1 node 0)
    rhs = 4.0 * np.pi * m1[:, None, None] * m1[None, :, None] * m1[None, None, :]
    # boundary values from the continuum potential
    N = p * n + 1
    idx = np.arange(N)
    I, J, K = np.meshgrid(idx, idx, idx, indexing='ij')
    onb = (I == 0) | (I == N - 1) | (J == 0) | (J == N - 1) | (K == 0) | (K == N - 1)
    Hb = np.zeros((N, N, N))
    pts = np.stack([x1[I[onb]], x1[J[onb]], x1[K[onb]]], axis=1)
    Hb[onb] = hat_potential_continuum(pts, ngl)
    r = rhs - stiffness_apply(K1, M1, Hb)
    r = r[1:-1, 1:-1, 1:-1]
    lam, V = scipy.linalg.eigh(K1[1:-1, 1:-1], M1[1:-1, 1:-1])   # V^T M V = I, V^T K V = diag(lam)
    rh = kron_apply(V.T, V.T, V.T, r)
    rh /= lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    H = Hb.copy()
    H[1:-1, 1:-1, 1:-1] = kron_apply(V, V, V, rh)
    return H, x1


def kept_table(p=3, half_width=8, ngl=8, keep=4):
    """Nodal values of H on [-keep, keep]^3 (the 8^3 elements around the vertex): ((2*keep*p+1),)*3."""
    H, x1 = basis_screen_table(p, half_width, ngl)
    s = p * (half_width - keep)
    e = p * (half_width + keep) + 1
    return H[s:e, s:e, s:e].copy()
