"""1-D Lagrange finite elements on equispaced nodes (oracle; test infrastructure).

The FE mesh solve of Sec. 2.2 uses order-p = q+2 tensor-product Lagrange
hexahedra on a uniform periodic mesh (Sec. 2, Fig. schematic).  On such a mesh
the 3-D stiffness and mass matrices are Kronecker products of the 1-D ones,
so everything here is 1-D.  Node placement is equispaced (the paper does not
state it; equispaced Lagrange nodes are the reading used throughout).
Integrals use Gauss-Legendre quadrature with enough points to be exact.
"""
import numpy as np


def gauss_legendre01(n):
    """n-point Gauss-Legendre rule mapped to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gll_nodes01(p):
    """Gauss-Lobatto-Legendre nodes on [0, 1]: the end points and the roots of P_p'."""
    if p == 1:
        return np.array([0.0, 1.0])
    x = np.sort(np.real(np.polynomial.legendre.Legendre.basis(p).deriv().roots()))
    return np.concatenate([[0.0], 0.5 * (x + 1.0), [1.0]])


def node_set(p, nodes=None):
    """The order-p nodes on [0, 1]: equispaced (None or 'equispaced') or 'gll'."""
    if nodes is None or nodes == 'equispaced':
        return np.linspace(0.0, 1.0, p + 1)
    if nodes == 'gll':
        return gll_nodes01(p)
    raise ValueError(nodes)


def lagrange_values(p, t, nodes=None):
    """Order-p Lagrange basis on [0,1] at points t: shape t.shape+(p+1,); equispaced nodes
    unless nodes = 'gll'."""
    nodes = node_set(p, nodes)
    t = np.asarray(t, dtype=np.float64)
    out = np.ones(t.shape + (p + 1,))
    for k in range(p + 1):
        for j in range(p + 1):
            if j != k:
                out[..., k] *= (t - nodes[j]) / (nodes[k] - nodes[j])
    return out


def lagrange_derivs(p, t):
    """d/dt of the equispaced order-p Lagrange basis on [0,1] (product rule)."""
    nodes = np.linspace(0.0, 1.0, p + 1)
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros(t.shape + (p + 1,))
    for k in range(p + 1):
        for m in range(p + 1):
            if m == k:
                continue
            term = np.full(t.shape, 1.0 / (nodes[k] - nodes[m]))
            for j in range(p + 1):
                if j != k and j != m:
                    term = term * (t - nodes[j]) / (nodes[k] - nodes[j])
            out[..., k] += term
    return out


def element_matrices(p, h, q=None, qnodes=None):
    """Element mass h*int(l_i l_j), stiffness (1/h)*int(l_i' l_j') on [0,1];
    with q given, also the mixed mass h*int(l^p_i l^q_j) (order-p rows, order-q columns,
    the order-q basis on the node set qnodes)."""
    t, w = gauss_legendre01(p + 2)
    L = lagrange_values(p, t)
    D = lagrange_derivs(p, t)
    Me = h * np.einsum('g,gi,gj->ij', w, L, L)
    Ke = (1.0 / h) * np.einsum('g,gi,gj->ij', w, D, D)
    if q is None:
        return Me, Ke
    Lq = lagrange_values(q, t, qnodes)
    Mpq = h * np.einsum('g,gi,gj->ij', w, L, Lq)
    return Me, Ke, Mpq


def assemble_periodic(Ae, n, rows_per_el, cols_per_el=None):
    """Periodic global assembly of an element matrix over n elements.

    Element e's local row k maps to global row (rows_per_el*e + k) mod (rows_per_el*n);
    likewise for columns (so a square order-p matrix uses rows_per_el = cols_per_el = p)."""
    if cols_per_el is None:
        cols_per_el = rows_per_el
    nr, nc = rows_per_el * n, cols_per_el * n
    A = np.zeros((nr, nc))
    for e in range(n):
        for i in range(Ae.shape[0]):
            for j in range(Ae.shape[1]):
                A[(rows_per_el * e + i) % nr, (cols_per_el * e + j) % nc] += Ae[i, j]
    return A


def assemble_open(Ae, n, p):
    """Non-periodic assembly on n elements: (p*n+1) x (p*n+1) nodes (used for Dirichlet boxes)."""
    N = p * n + 1
    A = np.zeros((N, N))
    for e in range(n):
        s = p * e
        A[s:s + p + 1, s:s + p + 1] += Ae
    return A


def periodic_matrices(p, n, h, q=1, qnodes=None):
    """1-D periodic order-p mass M1, stiffness K1 (p*n square) and mixed mass Mpq (p*n x q*n)."""
    Me, Ke, Mpq_e = element_matrices(p, h, q, qnodes)
    M1 = assemble_periodic(Me, n, p)
    K1 = assemble_periodic(Ke, n, p)
    Mpq = assemble_periodic(Mpq_e, n, p, q)
    return M1, K1, Mpq


def node_integrals_periodic(p, n, h):
    """w_k = integral of the k-th periodic global order-p basis function (row sums of M1)."""
    t, w = gauss_legendre01(p + 2)
    we = h * np.einsum('g,gi->i', w, lagrange_values(p, t))
    out = np.zeros(p * n)
    for e in range(n):
        for i in range(p + 1):
            out[(p * e + i) % (p * n)] += we[i]
    return out
