"""FE-P3M on the box [0, L]^3 with Neumann data dPhi/dn = g on its boundary, plain FP64
on the CPU (oracle; test infrastructure).

Sec. "Alternate boundary conditions": as for Dirichlet data (Eq. bcadjust), the mesh
problem takes the boundary data less what the short-range potential already carries,
dPhi^sm/dn = g - dPhi^sr/dn, so that dPhi/dn = g; the fully Neumann problem fixes the
additive constant separately.  In the Galerkin form the Neumann data is a boundary load:

    K phi = b + s,   s_m = int_{dV} (g - dPhi^sr/dn) v_m dS,

with b the screen load of oracle.dirichlet (the box integral of the screens).  Readings
(the paper gives only the principle):
  * n is the outward normal; Phi^sr near the boundary, its block and the table form are
    those of oracle.dirichlet (a point on a face takes the element the binning gives it);
  * the surface integral uses tensor Gauss-Legendre points on each face element: the
    integrand g - dPhi^sr/dn is smooth there, since every charge close to a face point is
    in that point's block and its 1/R part cancels (adjust=False keeps it, for
    comparison only);
  * the constant: K is singular (constant null space); the load is made compatible by
    removing its component along the node integrals (the periodic method's
    neutralisation), the constant mode is dropped (int phi^sm = 0), and potentials are
    compared up to a constant.
"""
import numpy as np
import scipy.linalg

from . import fe1d, screens, tables
from .dirichlet import P, Q_SCREEN, bin_box, element_coefficients, evaluate_mesh, open_matrices, short_range, \
    vertex_density
from .fep3m import corner


def short_range_normal_derivative(points, normal, pelem, ptloc, bins, Q, n, n_sr):
    """d/dn of Phi^sr at points (M, 3) on the boundary (outward unit normals (M, 3)), the
    points lying in elements pelem at local coordinates ptloc: the singular terms
    Q_j / |x - x_j| of the (cut-off) block and the gradients of the block's screen
    potentials through the table (order-3 element basis and its derivative)."""
    h = bins['h']
    keep = n_sr + 1
    Hk = tables.kept_table(P, half_width=keep + 4, keep=keep)
    lv = [fe1d.lagrange_values(P, ptloc[:, a]) for a in range(3)]
    ld = [fe1d.lagrange_derivs(P, ptloc[:, a]) / h for a in range(3)]
    c = screens.screen_coefficients(Q_SCREEN, h, bins['delta'])
    out = np.zeros(len(points))
    for j in range(len(Q)):
        d = bins['c3'][j] - pelem
        inb = np.all(np.abs(d) <= n_sr, axis=1)
        if Q[j] == 0 or not inb.any():
            continue
        m = np.flatnonzero(inb)
        rel = points[m] - bins['pos'][j]
        R = np.linalg.norm(rel, axis=1)
        val = -Q[j] * np.einsum('mk,mk->m', rel, normal[m]) / R ** 3      # d/dn of Q_j / |x - x_j|
        for kap in range(8):
            base = P * (-d[m] - corner(kap) + keep)
            g = np.zeros((len(m), 3))
            for mx in range(P + 1):
                for my in range(P + 1):
                    for mz in range(P + 1):
                        Hv = Hk[base[:, 0] + mx, base[:, 1] + my, base[:, 2] + mz]
                        g[:, 0] += Hv * ld[0][m, mx] * lv[1][m, my] * lv[2][m, mz]
                        g[:, 1] += Hv * lv[0][m, mx] * ld[1][m, my] * lv[2][m, mz]
                        g[:, 2] += Hv * lv[0][m, mx] * lv[1][m, my] * ld[2][m, mz]
            val -= Q[j] * c[j, kap] * (h * h) * np.einsum('mk,mk->m', g, normal[m])
        out[m] += val
    return out


def boundary_load(n, h, L, integrand, ngl):
    """s_m = int_{dV} f v_m dS over the six faces, f = integrand(points, normals, elements,
    local coordinates) evaluated once on every quadrature point: tensor Gauss-Legendre on
    each face element, accumulated at the face element's order-3 nodes."""
    N = P * n + 1
    s = np.zeros((N, N, N))
    t, w = fe1d.gauss_legendre01(ngl)
    T1, T2 = [x.ravel() for x in np.meshgrid(t, t, indexing='ij')]
    W = (w[:, None] * w[None, :]).ravel() * h * h
    l1 = fe1d.lagrange_values(P, T1)
    l2 = fe1d.lagrange_values(P, T2)
    G = len(W)
    E1, E2 = [x.ravel() for x in np.meshgrid(np.arange(n), np.arange(n), indexing='ij')]
    faces = []                                   # (axis, side, a1, a2) in point order
    pts, nrms, els, locs = [], [], [], []
    for ax in range(3):
        a1, a2 = (ax + 1) % 3, (ax + 2) % 3
        for side in (0, 1):
            el = np.zeros((n * n, G, 3), dtype=np.int64)
            el[..., ax] = n - 1 if side else 0
            el[..., a1] = E1[:, None]
            el[..., a2] = E2[:, None]
            loc = np.zeros((n * n, G, 3))
            loc[..., ax] = float(side)
            loc[..., a1] = T1[None, :]
            loc[..., a2] = T2[None, :]
            nrm = np.zeros(3)
            nrm[ax] = 1.0 if side else -1.0
            faces.append((ax, side, a1, a2))
            els.append(el.reshape(-1, 3))
            locs.append(loc.reshape(-1, 3))
            pts.append(((el + loc) * h).reshape(-1, 3))
            nrms.append(np.tile(nrm, (n * n * G, 1)))
    f = integrand(np.concatenate(pts), np.concatenate(nrms), np.concatenate(els), np.concatenate(locs))
    f = f.reshape(6, n * n, G) * W
    for k, (ax, side, a1, a2) in enumerate(faces):
        vals = np.einsum('eg,gi,gj->eij', f[k], l1, l2)            # [face element, node along a1, node along a2]
        for fe_, (e1, e2) in enumerate(zip(E1, E2)):
            idx = [None, None, None]
            idx[ax] = np.array([P * n if side else 0])
            idx[a1] = P * e1 + np.arange(P + 1)
            idx[a2] = P * e2 + np.arange(P + 1)
            view = vals[fe_] if a1 < a2 else vals[fe_].T              # order the two face axes
            s[np.ix_(idx[0], idx[1], idx[2])] += view.reshape(len(idx[0]), len(idx[1]), len(idx[2]))
    return s


def solve_compatible(rhs, M1, K1):
    """The fully Neumann Galerkin problem K phi = rhs on all nodes, K = K1 (x) M1 (x) M1 +
    M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1 (constant null space): the load less its component
    along the node integrals, the constant mode dropped (int phi = 0); exact, by fast
    diagonalisation."""
    w1 = M1.sum(axis=1)
    w3 = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
    rhs = rhs - rhs.sum() * w3 / w3.sum()                              # compatible load
    lam, V = scipy.linalg.eigh(K1, M1)
    rh = tables.kron_apply(V.T, V.T, V.T, rhs)
    D = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    z = int(np.argmin(np.abs(lam)))
    D[z, z, z] = np.inf                                                 # the constant mode
    return tables.kron_apply(V, V, V, rh / D)


def forward(pos, Q, L, n, gn, n_sr=3, adjust=True, ngl=8):
    """Phi_i at the charges (up to a constant) for Neumann data gn(points, normals), with
    the intermediates.  adjust=False takes dPhi^sm/dn = g instead."""
    Q = np.asarray(Q, dtype=np.float64)
    assert n >= 2 * n_sr + 1
    bins = bin_box(pos, L, n)
    h = bins['h']
    C = element_coefficients(bins, Q, n)
    r = vertex_density(C, n)
    M1, K1, Mpq = open_matrices(n, h)
    b = 4.0 * np.pi * tables.kron_apply(Mpq, Mpq, Mpq, r)

    def integrand(pts, nrm, el, loc):
        f = gn(pts, nrm)
        if adjust:
            f = f - short_range_normal_derivative(pts, nrm, el, loc, bins, Q, n, n_sr)
        return f

    s = boundary_load(n, h, L, integrand, ngl)
    phi_mesh = solve_compatible(b + s, M1, K1)
    phi_sm = evaluate_mesh(phi_mesh, bins['pos'], L, n)
    t = bins['delta'] / h + 0.5
    phi_sr = short_range(bins['pos'], bins['c3'], t, bins, Q, n, n_sr, exclude=np.arange(len(Q)))
    return dict(phi=phi_sm + phi_sr, phi_sm=phi_sm, phi_sr=phi_sr, phi_mesh=phi_mesh, b=b, s=s, bins=bins)
