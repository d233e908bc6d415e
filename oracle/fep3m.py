"""The finite-element P3M method, plain FP64 on the CPU (oracle; test infrastructure).

Follows Algorithm 1 step by step for the periodic cube [0, L)^3, screens of
order q = 1 and the order p = q + 2 = 3 FE mesh solve:

  1. bin: element of each charge and its offset delta from the element centre
     (Sec. 2.1, Fig. schematic; Sec. 3.1.1 "identify element, offsets");
  2. screens: c_kappa(delta) from Eq. moment1d / Eq. oned, aggregated per element
     into the element-to-point list C[e, kappa] = sum_{j in e} Q_j c_kappa(delta_j)
     (Sec. 3.1.2, "combined list of Q_i c_i");
  3. charge assignment onto the order-q mesh (Eq. assign, Eq. defineassign) and the
     FE load vector b_m = 4 pi int rho u_m = 4 pi (Mpq (x) Mpq (x) Mpq) r;
  4. mesh solve K phi = b (Sec. 2.2), K the periodic order-p stiffness, solved
     exactly here by fast diagonalisation; constant fixed by int phi = 0 (Sec. 4);
  5. smooth potential at the charges, Eq. evalsmooth;
  6. short-range potential, Sec. 2.4: the singular sum of Q_j/R over the
     (2 n_sr + 1)^3-element block around the target's element minus the screen
     potentials of all charges of that block, own screen included (Sec. 2.5),
     evaluated through the FE basis-screen table (Eq. sc, Remark of Sec. 4);
  7. Phi_i = Phi^sm_i + Phi^sr_i and U = 1/2 sum Q_i Phi_i (Eq. potentialenergy).

The adjoint (vjp) differentiates exactly this discrete U.  Readings of points
the paper leaves open: Poisson with 4 pi (Gaussian units, so Phi = Q/R);
half-open elements [c h, (c+1) h); block = cube of elements around the target's
element; tables per vertex hat (see oracle.tables); equispaced Lagrange nodes.
"""
import itertools

import numpy as np
import scipy.linalg

from . import fe1d, screens, tables

P_ORDER = 3   # p = q + 2 for q = 1 (Sec. 2, "basis functions of order p = q+2")
Q_ORDER = 1


def bin_particles(pos, L, n):
    """Element of each charge and its offset from the element centre.

    Wrap x -> x - L floor(x / L) (a result equal to L becomes 0); element
    c = floor(x * (n / L)) per axis (clamped to n-1); delta = x - (c + 1/2) h.
    Sorted order is stable by original index within an element."""
    pos = np.asarray(pos, dtype=np.float64)
    h = L / n
    inv_h = n / L
    xw = pos - L * np.floor(pos / L)
    xw[xw >= L] = 0.0
    c3 = np.floor(xw * inv_h).astype(np.int64)
    c3 = np.clip(c3, 0, n - 1)
    delta = xw - (c3 + 0.5) * h
    cell = c3[:, 0] + n * c3[:, 1] + n * n * c3[:, 2]
    perm = np.argsort(cell, kind='stable')
    count = np.bincount(cell, minlength=n ** 3)
    start = np.concatenate([[0], np.cumsum(count)[:-1]])
    return dict(h=h, c3=c3, cell=cell, delta=delta, perm=perm, start=start, count=count)


def element_coefficients(bins, Q, n):
    """C[e, kappa] = sum_{j in e} Q_j c_kappa(delta_j), shape (n^3, 8), units charge/h^3."""
    c = screens.screen_coefficients(Q_ORDER, bins['h'], bins['delta'])
    C = np.zeros((n ** 3, c.shape[1]))
    np.add.at(C, bins['cell'], np.asarray(Q)[:, None] * c)
    return C


def corner(kappa):
    """kappa = i + 2 j + 4 k -> (i, j, k): the element's corner vertex offsets."""
    return np.array([kappa & 1, (kappa >> 1) & 1, (kappa >> 2) & 1])


def vertex_density(C, n):
    """Order-1 nodal screen density r_v = sum over (element, corner) at vertex v (Eq. assign).

    Element (ex, ey, ez) has corner kappa at vertex (ex + i, ey + j, ez + k) mod n.
    Returns r indexed [vx, vy, vz]."""
    Cg = C.reshape(n, n, n, 8)          # [ez, ey, ex, kappa] (linear id ex + n ey + n^2 ez)
    r = np.zeros((n, n, n))             # [vx, vy, vz]
    for kap in range(8):
        i, j, k = corner(kap)
        # element (ex,ey,ez) -> vertex (ex+i, ey+j, ez+k)
        contrib = np.transpose(Cg[..., kap], (2, 1, 0))   # [ex, ey, ez]
        r += np.roll(contrib, shift=(i, j, k), axis=(0, 1, 2))
    return r


class MeshOperators:
    """1-D periodic order-p matrices for the mesh solve and its exact inverse."""

    def __init__(self, L, n, p=P_ORDER, q=Q_ORDER, qnodes=None):
        self.L, self.n, self.p, self.h = L, n, p, L / n
        self.M1, self.K1, self.Mpq = fe1d.periodic_matrices(p, n, self.h, q, qnodes)
        self.w1 = fe1d.node_integrals_periodic(p, n, self.h)
        lam, V = scipy.linalg.eigh(self.K1, self.M1)
        self.lam, self.V = lam, V
        self.null = int(np.argmin(np.abs(lam)))

    def w3(self):
        w = self.w1
        return w[:, None, None] * w[None, :, None] * w[None, None, :]

    def load_vector(self, r):
        """b = 4 pi (Mpq (x) Mpq (x) Mpq) r: b_m = 4 pi int rho u_m (Sec. 2.2, Eq. poisson with 4 pi)."""
        return 4.0 * np.pi * tables.kron_apply(self.Mpq, self.Mpq, self.Mpq, r)

    def neutralise(self, b):
        """b - (sum b) w / sum w: the load of a uniform background that cancels the net charge."""
        w3 = self.w3()
        return b - b.sum() * w3 / w3.sum()

    def apply_K(self, X):
        return tables.stiffness_apply(self.K1, self.M1, X)

    def solve(self, b):
        """phi with K phi = b (b neutral) and int phi = 0, by fast diagonalisation.

        V^T M1 V = I, V^T K1 V = diag(lam): K^-1 = (V(x)V(x)V) D^-1 (V(x)V(x)V)^T with
        D = lam_i + lam_j + lam_k; the constant mode (D = 0) is dropped, which is the
        int phi = 0 solution (its M-weighted component vanishes)."""
        V = self.V
        bh = tables.kron_apply(V.T, V.T, V.T, b)
        D = self.lam[:, None, None] + self.lam[None, :, None] + self.lam[None, None, :]
        D[self.null, self.null, self.null] = np.inf
        return tables.kron_apply(V, V, V, bh / D)

    def vertex_adjoint(self, lam):
        """mu = 4 pi (Mpq^T (x) Mpq^T (x) Mpq^T) lam on the vertex grid (transpose of load_vector)."""
        T = self.Mpq.T
        return 4.0 * np.pi * tables.kron_apply(T, T, T, lam)


def q3_basis(bins, p=P_ORDER):
    """u_m(x_i) for the 64 order-p basis functions of each charge's element, and their x-gradients.

    Local coordinate t = delta/h + 1/2 in [0, 1); m = mx + 4 my + 16 mz.
    Returns U (N, 64), G (N, 64, 3)."""
    h = bins['h']
    t = bins['delta'] / h + 0.5
    lv = [fe1d.lagrange_values(p, t[:, a]) for a in range(3)]
    ld = [fe1d.lagrange_derivs(p, t[:, a]) / h for a in range(3)]
    U = np.einsum('nk,nj,ni->nkji', lv[2], lv[1], lv[0]).reshape(-1, (p + 1) ** 3)
    G = np.stack([
        np.einsum('nk,nj,ni->nkji', lv[2], lv[1], ld[0]).reshape(-1, (p + 1) ** 3),
        np.einsum('nk,nj,ni->nkji', lv[2], ld[1], lv[0]).reshape(-1, (p + 1) ** 3),
        np.einsum('nk,nj,ni->nkji', ld[2], lv[1], lv[0]).reshape(-1, (p + 1) ** 3)], axis=2)
    return U, G


def element_node_index(c3, n, p=P_ORDER):
    """Global node indices (ix, iy, iz) of the 64 nodes of each element, m = mx + 4 my + 16 mz."""
    m = np.arange((p + 1) ** 3)
    mx, my, mz = m % (p + 1), (m // (p + 1)) % (p + 1), m // (p + 1) ** 2
    N = p * n
    ix = (p * c3[:, 0:1] + mx[None, :]) % N
    iy = (p * c3[:, 1:2] + my[None, :]) % N
    iz = (p * c3[:, 2:3] + mz[None, :]) % N
    return ix, iy, iz


def block_offsets(n_sr):
    r = range(-n_sr, n_sr + 1)
    return np.array([(dx, dy, dz) for dz in r for dy in r for dx in r])


def screen_window_matrix(n_sr, p=P_ORDER):
    """W[(d, kappa), m]: nodal value, at node m of the target element, of the table of the
    vertex hat at corner kappa of the source element at offset d from the target.

    The target element sits at -d - corner(kappa) (element units) from that vertex, so
    node m is at -d - corner + m/p; the kept table starts at -(n_sr + 1) with step 1/p."""
    keep = n_sr + 1
    Hk = tables.kept_table(p, half_width=keep + 4, keep=keep)
    offs = block_offsets(n_sr)
    m = np.arange((p + 1) ** 3)
    mx, my, mz = m % (p + 1), (m // (p + 1)) % (p + 1), m // (p + 1) ** 2
    W = np.zeros((len(offs), 8, (p + 1) ** 3))
    for k, d in enumerate(offs):
        for kap in range(8):
            rel = -d - corner(kap)          # target element relative to the vertex
            base = p * (rel + keep)
            W[k, kap] = Hk[base[0] + mx, base[1] + my, base[2] + mz]
    return W.reshape(len(offs) * 8, (p + 1) ** 3)


def gather_block_coefficients(C, c3, n, offs):
    """Cblk[i, (d, kappa)] = C[(e_i + d) mod n, kappa] for each target i."""
    src = (c3[:, None, :] + offs[None, :, :]) % n
    s = src[..., 0] + n * src[..., 1] + n * n * src[..., 2]
    return C[s].reshape(len(c3), -1)


def singular_sums(bins, Q, n, n_sr, weights=None):
    """Sum over j != i in the block of weights_j / R_ij and of weights_j (x_j - x_i)/R^3.

    weights defaults to Q (the potential); the adjoint passes its own weights."""
    if weights is None:
        weights = Q
    h, c3, delta = bins['h'], bins['c3'], bins['delta']
    perm, start, count = bins['perm'], bins['start'], bins['count']
    N = len(Q)
    phi = np.zeros(N)
    grad = np.zeros((N, 3))
    idx = np.arange(N)
    for d in block_offsets(n_sr):
        src = (c3 + d) % n
        s = src[:, 0] + n * src[:, 1] + n * n * src[:, 2]
        cnt = count[s]
        for k in range(int(cnt.max()) if N else 0):
            valid = k < cnt
            j = perm[np.where(valid, start[s] + k, 0)]
            valid &= j != idx
            rel = d * h + delta[j] - delta                      # x_j - x_i (block image)
            R = np.sqrt(np.einsum('nk,nk->n', rel, rel))
            R = np.where(valid, R, 1.0)
            wj = np.where(valid, weights[j], 0.0)
            phi += wj / R
            grad += (wj / R ** 3)[:, None] * rel                # d/dx_i of w_j / |x_j - x_i|
    return phi, grad


def forward(pos, Q, L, n, n_sr=3, neutralise=True, chunk=4096, want_grad=False, targets=None):
    """Phi_i and U for charges Q at pos (N x 3), with all intermediates (Algorithm 1).

    targets (optional index array): evaluate Phi only at these charges (the mesh
    solve still uses every charge); then phi and its parts have len(targets)
    entries and U is not formed."""
    pos = np.asarray(pos, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    assert n >= 2 * n_sr + 1, "the short-range block must not wrap onto itself"
    bins = bin_particles(pos, L, n)
    h = bins['h']
    C = element_coefficients(bins, Q, n)
    r = vertex_density(C, n)
    ops = MeshOperators(L, n)
    b = ops.load_vector(r)
    if neutralise:
        b = ops.neutralise(b)
    phi_mesh = ops.solve(b)
    if targets is not None:
        return _forward_targets(bins, C, Q, n, n_sr, phi_mesh, np.asarray(targets), chunk)
    U3, G3 = q3_basis(bins)
    ix, iy, iz = element_node_index(bins['c3'], n)
    phi_nodes = phi_mesh[ix, iy, iz]                            # (N, 64)
    phi_sm = np.einsum('nm,nm->n', phi_nodes, U3)
    phi_sing, grad_sing = singular_sums(bins, Q, n, n_sr)
    Wmat = screen_window_matrix(n_sr)
    offs = block_offsets(n_sr)
    phi_scr = np.zeros(len(Q))
    grad_field = np.zeros((len(Q), 3))
    for s0 in range(0, len(Q), chunk):
        sl = slice(s0, s0 + chunk)
        Cblk = gather_block_coefficients(C, bins['c3'][sl], n, offs)
        Gscr = (h * h) * (Cblk @ Wmat)                          # screen field at the 64 nodes
        phi_scr[sl] = np.einsum('nm,nm->n', Gscr, U3[sl])
        if want_grad:
            grad_field[sl] = np.einsum('nm,nmk->nk', phi_nodes[sl] - Gscr, G3[sl])
    phi = phi_sm + phi_sing - phi_scr
    U = 0.5 * np.dot(Q, phi)
    out = dict(phi=phi, U=U, bins=bins, C=C, r=r, b=b, phi_mesh=phi_mesh, phi_sm=phi_sm,
               phi_sing=phi_sing, phi_scr=phi_scr, ops=ops, Wmat=Wmat, U3=U3, G3=G3)
    if want_grad:
        out['grad_field'] = grad_field + grad_sing              # d/dx of (sum_j Q_j K(x, j)) at x_i
    return out


def _forward_targets(bins, C, Q, n, n_sr, phi_mesh, tg, chunk):
    """Phi at the charges tg only: the same three parts as forward(), restricted."""
    h = bins['h']
    sub = dict(bins)
    for k in ('c3', 'cell', 'delta'):
        sub[k] = bins[k][tg]
    U3, _ = q3_basis(sub)
    ix, iy, iz = element_node_index(sub['c3'], n)
    phi_sm = np.einsum('nm,nm->n', phi_mesh[ix, iy, iz], U3)
    # singular sums with the targets' own indices excluded
    phi_sing = np.zeros(len(tg))
    perm, start, count = bins['perm'], bins['start'], bins['count']
    for d in block_offsets(n_sr):
        src = (sub['c3'] + d) % n
        s = src[:, 0] + n * src[:, 1] + n * n * src[:, 2]
        cnt = count[s]
        for k in range(int(cnt.max()) if len(tg) else 0):
            valid = k < cnt
            j = perm[np.where(valid, start[s] + k, 0)]
            valid &= j != tg
            rel = d * h + bins['delta'][j] - sub['delta']
            R = np.where(valid, np.sqrt(np.einsum('nk,nk->n', rel, rel)), 1.0)
            phi_sing += np.where(valid, Q[j], 0.0) / R
    Wmat = screen_window_matrix(n_sr)
    offs = block_offsets(n_sr)
    phi_scr = np.zeros(len(tg))
    for s0 in range(0, len(tg), chunk):
        sl = slice(s0, s0 + chunk)
        Cblk = gather_block_coefficients(C, sub['c3'][sl], n, offs)
        phi_scr[sl] = np.einsum('nm,nm->n', (h * h) * (Cblk @ Wmat), U3[sl])
    return dict(phi=phi_sm + phi_sing - phi_scr, phi_sm=phi_sm, phi_sing=phi_sing, phi_scr=phi_scr,
                phi_mesh=phi_mesh, bins=bins, C=C)


def vjp(fwd, Q, gU=1.0, gphi=None, n_sr=3, chunk=4096):
    """Reverse sweep of forward(): returns (dL/dpos (N,3), dL/dQ (N,)) for L = gU U + gphi . Phi.

    With w_i = gU Q_i / 2 + gphi_i and Phi_t = sum_j Q_j K(t, j):
      dL/dQ_i = gU Phi_i / 2 + sum_t w_t K(t, i),
      dL/dx_i = w_i d/dx_i [sum_j Q_j K(x_i, j)] + Q_i d/dx_i [sum_t w_t K(t, i)].
    The kernel K(t, i) has three parts, each differentiated here:
      singular 1/R over the block (symmetric);
      screen  -sum_kappa c_kappa(delta_i) h^2 T_kappa(x_t)  (source side through c, target side through T);
      mesh    u(x_t)^T S 4 pi Mpq c(delta_i) with S the symmetric solve operator, so the
              source side needs lam = S g, g = sum_t w_t u(x_t) (one more mesh solve)."""
    bins, ops, C = fwd['bins'], fwd['ops'], fwd['C']
    n, h = ops.n, bins['h']
    Q = np.asarray(Q, dtype=np.float64)
    N = len(Q)
    w = 0.5 * gU * Q + (0.0 if gphi is None else np.asarray(gphi, dtype=np.float64))
    if 'grad_field' not in fwd:
        raise ValueError("forward(..., want_grad=True) is required")
    dx = w[:, None] * fwd['grad_field']
    # singular, source side
    psi_sing, grad_w = singular_sums(bins, Q, n, n_sr, weights=w)
    dx += Q[:, None] * grad_w
    dQ = 0.5 * gU * fwd['phi'] + psi_sing
    # screen, source side: A[s, kappa] = sum_t w_t h^2 T_kappa(x_t) over targets t whose block holds s
    offs = block_offsets(n_sr)
    A = np.zeros((n ** 3, 8))
    Wmat, U3 = fwd['Wmat'], fwd['U3']
    for s0 in range(0, N, chunk):
        sl = slice(s0, s0 + chunk)
        vals = (h * h) * w[sl, None] * (U3[sl] @ Wmat.T)        # (n_t, 343*8)
        src = (bins['c3'][sl, None, :] + offs[None, :, :]) % n
        s = src[..., 0] + n * src[..., 1] + n * n * src[..., 2]
        np.add.at(A, (np.repeat(s, 8, axis=1).ravel(), np.tile(np.arange(8), s.size)), vals.ravel())
    # mesh, source side: g = sum_t w_t u(x_t); lam = S g; mu = 4 pi Mpq^T lam at the vertices
    ix, iy, iz = element_node_index(bins['c3'], n)
    g = np.zeros((3 * n,) * 3)
    np.add.at(g, (ix.ravel(), iy.ravel(), iz.ravel()), (w[:, None] * U3).ravel())
    g = ops.neutralise(g)
    lam = ops.solve(g)
    mu = ops.vertex_adjoint(lam)                                 # [vx, vy, vz]
    # per charge: sum_kappa (mu at its corner vertex - A[e, kappa]) times c and grad c
    c = screens.screen_coefficients(Q_ORDER, h, bins['delta'])  # (N, 8), 1/h^3
    dc = screen_coefficient_gradients(h, bins['delta'])         # (N, 8, 3)
    coef = np.zeros((N, 8))
    for kap in range(8):
        v = (bins['c3'] + corner(kap)) % n
        coef[:, kap] = mu[v[:, 0], v[:, 1], v[:, 2]] - A[bins['cell'], kap]
    dQ += np.einsum('nk,nk->n', coef, c)
    dx += Q[:, None] * np.einsum('nk,nkd->nd', coef, dc)
    return dx, dQ, dict(A=A, g=g, lam=lam, mu=mu)


def screen_coefficient_gradients(h, delta):
    """d c_kappa / d x for q = 1, by differentiating the solved weights of Eq. moment1d.

    The weights are affine in delta (solution of a fixed linear system with right-hand
    side (1, delta)), so the derivative is the solve with right-hand side (0, 1)."""
    Om = screens.moment_matrix_1d(Q_ORDER, h)
    dw = np.linalg.solve(Om, np.array([0.0, 1.0]))             # d w_i / d delta
    w = [screens.screen_weights_1d(Q_ORDER, h, delta[:, a]) for a in range(3)]
    out = np.zeros((len(delta), 8, 3))
    for kap in range(8):
        i, j, k = corner(kap)
        out[:, kap, 0] = dw[i] * w[1][:, j] * w[2][:, k]
        out[:, kap, 1] = w[0][:, i] * dw[j] * w[2][:, k]
        out[:, kap, 2] = w[0][:, i] * w[1][:, j] * dw[k]
    return out


def forces_at(pos, Q, L, n, targets, n_sr=3, chunk=4096):
    """-dU/dx at the charges listed in targets only: the energy's adjoint (vjp with
    gU = 1, gphi = 0, weights w = Q / 2) restricted to those charges.

    The parts of vjp() are local to the target, except the mesh part: the
    potential's mesh solve and the adjoint mesh solve still take every charge.
    Target side (w_i grad_x [sum_j Q_j K(x, j)] at x_i): the singular sums over
    the target's block, and the gradient of (mesh potential - screen field) at
    the charge.  Source side (Q_i grad_x_i [sum_t w_t K(t, i)]): the singular sums
    with weights w, the screen adjoint A[e_i, kappa] = sum over the charges t
    whose block holds e_i of w_t h^2 T_kappa(x_t), and the vertex adjoint mu."""
    pos = np.asarray(pos, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    tg = np.asarray(targets)
    bins = bin_particles(pos, L, n)
    h = bins['h']
    C = element_coefficients(bins, Q, n)
    r = vertex_density(C, n)
    ops = MeshOperators(L, n)
    phi_mesh = ops.solve(ops.neutralise(ops.load_vector(r)))
    w = 0.5 * Q
    sub = dict(bins)
    for k in ('c3', 'cell', 'delta'):
        sub[k] = bins[k][tg]
    U3t, G3t = q3_basis(sub)
    offs = block_offsets(n_sr)
    Wmat = screen_window_matrix(n_sr)
    # target side: mesh potential minus the screen field, differentiated at the charge
    ix, iy, iz = element_node_index(sub['c3'], n)
    Cblk = gather_block_coefficients(C, sub['c3'], n, offs)
    Gscr = (h * h) * (Cblk @ Wmat)
    grad_field = np.einsum('nm,nmk->nk', phi_mesh[ix, iy, iz] - Gscr, G3t)
    # singular sums at the targets: sum_j Q_j (x_j - x_i)/R^3 and the same with w
    perm, start, count = bins['perm'], bins['start'], bins['count']
    grad_q = np.zeros((len(tg), 3))
    grad_w = np.zeros((len(tg), 3))
    for d in offs:
        src = (sub['c3'] + d) % n
        s = src[:, 0] + n * src[:, 1] + n * n * src[:, 2]
        cnt = count[s]
        for k in range(int(cnt.max()) if len(tg) else 0):
            valid = k < cnt
            j = perm[np.where(valid, start[s] + k, 0)]
            valid &= j != tg
            rel = d * h + bins['delta'][j] - sub['delta']
            R = np.where(valid, np.sqrt(np.einsum('nk,nk->n', rel, rel)), 1.0)
            grad_q += (np.where(valid, Q[j], 0.0) / R ** 3)[:, None] * rel
            grad_w += (np.where(valid, w[j], 0.0) / R ** 3)[:, None] * rel
    dx = w[tg, None] * (grad_field + grad_q) + Q[tg, None] * grad_w
    # screen, source side: A[e_i, kappa] over the charges t of the blocks that hold e_i
    # (t in element e_i - d for the block offset d; the window row of offset d)
    A = np.zeros((len(tg), 8))
    nw = Wmat.reshape(len(offs), 8, -1)
    for di, d in enumerate(offs):
        src = (sub['c3'] - d) % n
        s = src[:, 0] + n * src[:, 1] + n * n * src[:, 2]
        cnt = count[s]
        for k in range(int(cnt.max()) if len(tg) else 0):
            valid = k < cnt
            t = perm[np.where(valid, start[s] + k, 0)]
            Ut, _ = q3_basis(dict(h=h, delta=bins['delta'][t]))
            A += (h * h) * np.where(valid, w[t], 0.0)[:, None] * (Ut @ nw[di].T)
    # mesh, source side: lam = S g with g = sum_t w_t u(x_t) over every charge
    g = np.zeros((3 * n,) * 3)
    for s0 in range(0, len(Q), 1 << 18):
        sl = slice(s0, s0 + (1 << 18))
        U3, _ = q3_basis(dict(h=h, delta=bins['delta'][sl]))
        gx, gy, gz = element_node_index(bins['c3'][sl], n)
        np.add.at(g, (gx.ravel(), gy.ravel(), gz.ravel()), (w[sl, None] * U3).ravel())
    mu = ops.vertex_adjoint(ops.solve(ops.neutralise(g)))
    dc = screen_coefficient_gradients(h, sub['delta'])
    coef = np.zeros((len(tg), 8))
    for kap in range(8):
        v = (sub['c3'] + corner(kap)) % n
        coef[:, kap] = mu[v[:, 0], v[:, 1], v[:, 2]] - A[:, kap]
    dx += Q[tg, None] * np.einsum('nk,nkd->nd', coef, dc)
    return -dx
