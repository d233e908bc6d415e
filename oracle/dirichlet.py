"""FE-P3M on the box [0, L]^3 with Dirichlet data Phi = g on its boundary, plain FP64 on
the CPU (oracle; test infrastructure).

Sec. "Alternate boundary conditions": the periodic method carries over by adjusting the
mesh problem's boundary values for the short-range potential already present there,
Eq. bcadjust: Phi^sm = g - Phi^sr on the boundary, so that Phi = Phi^sm + Phi^sr = g.
Algorithm 1 marks the step ("adjust boundary conditions" for surface elements).  The
steps, for screens of order q = 1 and the order-3 mesh:

  1. bin the charges into the n^3 elements of the box (no wrapping);
  2. screens and element lists C[e, kappa] (Eq. oned, Eq. moment1d);
  3. vertex density r on the (n+1)^3 vertices and the load vector
     b = 4 pi (Mpq (x) Mpq (x) Mpq) r, integrated over the box only (the part of a
     boundary charge's screen outside the box does not enter the box's Poisson problem);
  4. boundary values Phi^sm = g - Phi^sr at the boundary nodes of the order-3 mesh;
  5. Dirichlet FE solve for the interior nodes, exact by fast diagonalisation;
  6. Phi_i = Phi^sm(x_i) + Phi^sr_i at the charges.

Readings (the paper states only Eq. bcadjust):
  * the short-range block of a point is the cube of (2 n_sr + 1)^3 elements around the
    point's element, cut off at the box faces (no images);
  * a boundary node's element follows the charge binning: c = min(floor(x / h), n - 1)
    per axis, so a node shared by several elements takes the lowest-index one;
  * Phi^sr at a point is the singular sum over the block's charges minus their screen
    potentials through the FE basis-screen table (Eq. sc, Remark of Sec. 4), the same
    table as the periodic oracle; at a node the table's nodal value is used directly.
"""
import numpy as np
import scipy.linalg

from . import fe1d, screens, tables
from .fep3m import block_offsets, corner

P = 3
Q_SCREEN = 1


def open_matrices(n, h):
    """Order-3 mass M1 and stiffness K1 on the 3n + 1 nodes of [0, n h], and the mixed mass
    Mpq ((3n + 1) x (n + 1)) against the order-1 vertex functions."""
    Me, Ke, Mpq_e = fe1d.element_matrices(P, h, Q_SCREEN)
    M1 = fe1d.assemble_open(Me, n, P)
    K1 = fe1d.assemble_open(Ke, n, P)
    Mpq = np.zeros((P * n + 1, n + 1))
    for e in range(n):
        Mpq[P * e:P * e + P + 1, e:e + 2] += Mpq_e
    return M1, K1, Mpq


def bin_box(pos, L, n):
    """Element and offset from its centre of each charge (0 <= x <= L), half-open elements."""
    pos = np.asarray(pos, dtype=np.float64)
    assert np.all((pos >= 0) & (pos <= L)), "charges must lie in the box"
    h = L / n
    c3 = np.clip(np.floor(pos * (n / L)).astype(np.int64), 0, n - 1)
    return dict(h=h, c3=c3, delta=pos - (c3 + 0.5) * h, pos=pos)


def element_coefficients(bins, Q, n):
    c = screens.screen_coefficients(Q_SCREEN, bins['h'], bins['delta'])
    C = np.zeros((n, n, n, 8))                  # [ex, ey, ez, kappa]
    c3 = bins['c3']
    np.add.at(C, (c3[:, 0], c3[:, 1], c3[:, 2]), np.asarray(Q)[:, None] * c)
    return C


def vertex_density(C, n):
    """r[vx, vy, vz] on the (n+1)^3 vertices: element (ex, ey, ez)'s corner kappa sits at
    vertex (ex + i, ey + j, ez + k)."""
    r = np.zeros((n + 1, n + 1, n + 1))
    for kap in range(8):
        i, j, k = corner(kap)
        r[i:i + n, j:j + n, k:k + n] += C[..., kap]
    return r


def short_range(points, pelem, ptloc, bins, Q, n, n_sr, exclude=None):
    """Phi^sr at points (M, 3) lying in elements pelem (M, 3) at local coordinates ptloc
    (M, 3) in [0, 1]: sum over the charges j of the (cut-off) block of Q_j / |x - x_j|
    minus Q_j times their screen potential, the table interpolated with the order-3
    element basis at ptloc.  exclude[m] = the charge whose singular term point m
    leaves out (its own); its screen is still subtracted (Sec. 2.5)."""
    h = bins['h']
    keep = n_sr + 1
    Hk = tables.kept_table(P, half_width=keep + 4, keep=keep)
    lv = [fe1d.lagrange_values(P, ptloc[:, a]) for a in range(3)]          # (M, 4) each
    c = screens.screen_coefficients(Q_SCREEN, h, bins['delta'])               # (N, 8), 1/h^3
    src_el = bins['c3']
    out = np.zeros(len(points))
    for j in range(len(Q)):
        d = src_el[j] - pelem                                                 # source minus point element
        inb = np.all(np.abs(d) <= n_sr, axis=1)
        if not inb.any():
            continue
        m = np.flatnonzero(inb)
        own = np.zeros(len(m), dtype=bool) if exclude is None else exclude[m] == j
        R = np.linalg.norm(points[m] - bins['pos'][j], axis=1)
        val = np.where(own, 0.0, Q[j] / np.where(own, 1.0, R))
        for kap in range(8):
            # point element relative to the vertex: -d - corner, table nodes in steps 1/3
            base = P * (-d[m] - corner(kap) + keep)
            tv = np.zeros(len(m))
            for mx in range(P + 1):
                for my in range(P + 1):
                    for mz in range(P + 1):
                        tv += (Hk[base[:, 0] + mx, base[:, 1] + my, base[:, 2] + mz]
                               * lv[0][m, mx] * lv[1][m, my] * lv[2][m, mz])
            val -= Q[j] * c[j, kap] * (h * h) * tv                             # h^2 H(x / h) per unit density
        out[m] += val
    return out


def boundary_nodes(n, h):
    """Indices, positions, elements and local coordinates of the boundary nodes of the
    order-3 mesh (3n + 1 nodes per axis)."""
    N = P * n + 1
    I, J, K = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing='ij')
    onb = (I == 0) | (I == N - 1) | (J == 0) | (J == N - 1) | (K == 0) | (K == N - 1)
    idx = np.stack([I[onb], J[onb], K[onb]], axis=1)
    el = np.minimum(idx // P, n - 1)
    return onb, idx * (h / P), el, idx / P - el


def solve_interior(b, phiB, M1, K1):
    """The Galerkin Dirichlet problem: K phi = b at the interior nodes with phi = phiB on
    the boundary nodes (phiB's interior entries zero), K = K1 (x) M1 (x) M1 + M1 (x) K1
    (x) M1 + M1 (x) M1 (x) K1; exact, by fast diagonalisation of the interior block."""
    rhs = b - (tables.kron_apply(K1, M1, M1, phiB) + tables.kron_apply(M1, K1, M1, phiB)
               + tables.kron_apply(M1, M1, K1, phiB))
    lam, V = scipy.linalg.eigh(K1[1:-1, 1:-1], M1[1:-1, 1:-1])
    rh = tables.kron_apply(V.T, V.T, V.T, rhs[1:-1, 1:-1, 1:-1])
    rh /= lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    phi_mesh = phiB.copy()
    phi_mesh[1:-1, 1:-1, 1:-1] = tables.kron_apply(V, V, V, rh)
    return phi_mesh


def forward(pos, Q, L, n, g, n_sr=3, adjust=True):
    """Phi_i at the charges for Dirichlet data g (a function of (M, 3) points), with the
    intermediates.  adjust=False sets Phi^sm = g on the boundary instead of Eq. bcadjust."""
    Q = np.asarray(Q, dtype=np.float64)
    assert n >= 2 * n_sr + 1
    bins = bin_box(pos, L, n)
    h = bins['h']
    C = element_coefficients(bins, Q, n)
    r = vertex_density(C, n)
    M1, K1, Mpq = open_matrices(n, h)
    b = 4.0 * np.pi * tables.kron_apply(Mpq, Mpq, Mpq, r)
    onb, bpts, bel, bloc = boundary_nodes(n, h)
    gb = g(bpts)
    if adjust:
        gb = gb - short_range(bpts, bel, bloc, bins, Q, n, n_sr)
    phiB = np.zeros(onb.shape)
    phiB[onb] = gb
    phi_mesh = solve_interior(b, phiB, M1, K1)
    # evaluation at the charges
    t = bins['delta'] / h + 0.5
    lv = [fe1d.lagrange_values(P, t[:, a]) for a in range(3)]
    c3 = bins['c3']
    phi_sm = np.zeros(len(Q))
    for mx in range(P + 1):
        for my in range(P + 1):
            for mz in range(P + 1):
                phi_sm += (phi_mesh[P * c3[:, 0] + mx, P * c3[:, 1] + my, P * c3[:, 2] + mz]
                           * lv[0][:, mx] * lv[1][:, my] * lv[2][:, mz])
    phi_sr = short_range(bins['pos'], c3, t, bins, Q, n, n_sr, exclude=np.arange(len(Q)))
    phi = phi_sm + phi_sr
    return dict(phi=phi, U=0.5 * np.dot(Q, phi), phi_sm=phi_sm, phi_sr=phi_sr, phi_mesh=phi_mesh,
                b=b, r=r, C=C, bins=bins)


def evaluate_mesh(phi_mesh, points, L, n):
    """Phi^sm at arbitrary points of the box from the nodal values (order-3 element basis)."""
    h = L / n
    points = np.asarray(points, dtype=np.float64)
    c3 = np.clip(np.floor(points / h).astype(np.int64), 0, n - 1)
    t = points / h - c3
    lv = [fe1d.lagrange_values(P, t[:, a]) for a in range(3)]
    out = np.zeros(len(points))
    for mx in range(P + 1):
        for my in range(P + 1):
            for mz in range(P + 1):
                out += (phi_mesh[P * c3[:, 0] + mx, P * c3[:, 1] + my, P * c3[:, 2] + mz]
                        * lv[0][:, mx] * lv[1][:, my] * lv[2][:, mz])
    return out
