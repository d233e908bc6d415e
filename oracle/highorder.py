"""FE-P3M with screens of any order q >= 1 and the order p = q + 2 mesh, plain FP64
on the CPU (oracle; test infrastructure).

The same steps as oracle.fep3m (Algorithm 1), written for a general screen order:

  1. bin the charges (Sec. 2.1; the binning of oracle.fep3m);
  2. screens (Eq. oned, Eq. moment1d): each charge carries c_kappa(delta) on the
     (q+1)^3 order-q nodes of its element; per element C[e, kappa] = sum Q_j c_kappa;
  3. charge assignment (Eq. assign): the element lists add into the nodal density r
     of the periodic order-q mesh (q n points per axis); load vector
     b = 4 pi (Mpq (x) Mpq (x) Mpq) r (Sec. 2.2);
  4. order-p mesh solve K phi = b, int phi = 0, by fast diagonalisation;
  5. smooth potential at the charges (Eq. evalsmooth);
  6. short range (Sec. 2.4, Eq. sc and the Remark of Sec. 4): singular sum over the
     block minus the screen potentials of the block's charges, through FE tables of
     the basis screens stored as order-p nodal values;
  7. Phi = Phi^sm + Phi^sr and U = 1/2 sum Q Phi (Eq. potentialenergy).

Readings beyond those of oracle.fep3m (the paper leaves them open):
  * the order-q screen basis uses Gauss-Lobatto-Legendre nodes (NODES below); the
    equispaced set stays available (nodes='equispaced');
  * the 1-D order-q nodal functions of the screen mesh come in q types: type 0, the
    vertex function (support the two elements next to its vertex), and types
    i = 1 .. q-1, the interior functions of one element (node at i/q of it).  A 3-D
    basis screen is a product of three 1-D types, and all basis screens of one type
    are translates of one function, so q^3 tables serve every basis screen (for
    q = 1 the single hat table of oracle.tables);
  * each table is anchored at the left vertex of the element that holds its node
    (the vertex itself for type 0).  Local node i of an element along an axis has
    anchor offset 1 if i = q (the next element's vertex) else 0, and type i mod q;
  * a table is the Dirichlet FE solution (order p, h = 1) on a box that extends
    half_width elements beyond the anchor on each side, and one element more on the
    right along axes of interior type, so that every box is symmetric about the
    centre of its basis screen's support; boundary values are the continuum
    potential (Eq. screenintegral) by tensor Gauss-Legendre quadrature on the
    polynomial pieces of the screen.
"""
import functools
import itertools

import numpy as np
import scipy.linalg

from . import fe1d, screens, tables
from .fep3m import MeshOperators, bin_particles, block_offsets, element_node_index, gather_block_coefficients, \
    q3_basis, singular_sums

# Node set of the order-q screen basis (the order-p mesh space does not depend on one).
# Gauss-Lobatto-Legendre: with it the error against Ewald on the paper's two-cube
# workload (Sec. 4) falls faster at each step of q through q = 4, as Fig. compareerr
# shows; with equispaced nodes the q = 4 screens are larger than the q = 3 ones at the
# block's edge and q = 4 loses to q = 3.  The two sets coincide for q <= 2.
NODES = 'gll'


def basis_pieces_1d(q, t, nodes=NODES):
    """Polynomial pieces (a, b, f) of the 1-D type-t order-q nodal function, element
    units, anchor at 0: type 0 on [-1, 0] and [0, 1], type t >= 1 on [0, 1]."""
    if t == 0:
        return [(-1.0, 0.0, lambda x: fe1d.lagrange_values(q, x + 1.0, nodes)[..., q]),
                (0.0, 1.0, lambda x: fe1d.lagrange_values(q, x, nodes)[..., 0])]
    return [(0.0, 1.0, lambda x, t=t: fe1d.lagrange_values(q, x, nodes)[..., t])]


def quadrature_1d(q, t, ngl, nodes=NODES):
    """Points and weights times the type-t nodal function, per polynomial piece."""
    tq, wq = fe1d.gauss_legendre01(ngl)
    xs, ws = [], []
    for (a, b, f) in basis_pieces_1d(q, t, nodes):
        x = a + (b - a) * tq
        xs.append(x)
        ws.append((b - a) * wq * f(x))
    return np.concatenate(xs), np.concatenate(ws)


def basis_potential_continuum(q, t3, points, ngl=8, nodes=NODES):
    """int psi_t(xi) / |x - xi| dxi for the 3-D basis screen of type t3 = (tx, ty, tz),
    anchor at the origin, h = 1 (Eq. screenintegral), points well outside its support."""
    q1 = [quadrature_1d(q, t, ngl, nodes) for t in t3]
    X, Y, Z = np.meshgrid(q1[0][0], q1[1][0], q1[2][0], indexing='ij')
    W = q1[0][1][:, None, None] * q1[1][1][None, :, None] * q1[2][1][None, None, :]
    return tables.coulomb_quadrature(points, np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel())


def mixed_mass_column(p, q, t, lo, nel, nodes=NODES):
    """int phi^p_k(x) psi_t(x) dx for the order-p nodes k of the open mesh of nel elements
    starting at x = lo (element units), psi_t anchored at 0."""
    _, _, Mpq_e = fe1d.element_matrices(p, 1.0, q, nodes)
    m1 = np.zeros(p * nel + 1)
    c = -lo                                     # the anchor is the left end of element c
    if t == 0:
        m1[p * (c - 1):p * c + 1] += Mpq_e[:, q]    # element left of the vertex: its last node
        m1[p * c:p * (c + 1) + 1] += Mpq_e[:, 0]    # element right of the vertex: its first node
    else:
        m1[p * c:p * (c + 1) + 1] += Mpq_e[:, t]
    return m1


def box_extent(t, half_width):
    """Element range [lo, hi) of a table's box along an axis of type t."""
    return -half_width, half_width + (1 if t else 0)


@functools.lru_cache(maxsize=256)
def type_table(p, q, t3, half_width=6, ngl=6, nodes=NODES):
    """FE potential of the basis screen of type t3 on its box (h = 1): H[ix, iy, iz] at
    x = lo_a + k / p along each axis a.  Galerkin: K_II H_I = 4 pi (Mpq psi)_I - K_IB H_B,
    solved exactly by fast diagonalisation of the 1-D Dirichlet pencils."""
    ext = [box_extent(t, half_width) for t in t3]
    nel = [hi - lo for (lo, hi) in ext]
    Me, Ke = fe1d.element_matrices(p, 1.0)
    M1 = [fe1d.assemble_open(Me, ne, p) for ne in nel]
    K1 = [fe1d.assemble_open(Ke, ne, p) for ne in nel]
    m1 = [mixed_mass_column(p, q, t, lo, ne, nodes) for t, (lo, _), ne in zip(t3, ext, nel)]
    rhs = 4.0 * np.pi * m1[0][:, None, None] * m1[1][None, :, None] * m1[2][None, None, :]
    x1 = [lo + np.arange(p * ne + 1) / p for (lo, _), ne in zip(ext, nel)]
    N = [len(x) for x in x1]
    I, J, K = np.meshgrid(np.arange(N[0]), np.arange(N[1]), np.arange(N[2]), indexing='ij')
    onb = (I == 0) | (I == N[0] - 1) | (J == 0) | (J == N[1] - 1) | (K == 0) | (K == N[2] - 1)
    Hb = np.zeros(tuple(N))
    pts = np.stack([x1[0][I[onb]], x1[1][J[onb]], x1[2][K[onb]]], axis=1)
    Hb[onb] = basis_potential_continuum(q, t3, pts, ngl, nodes)
    r = rhs - (tables.kron_apply(K1[0], M1[1], M1[2], Hb) + tables.kron_apply(M1[0], K1[1], M1[2], Hb)
               + tables.kron_apply(M1[0], M1[1], K1[2], Hb))
    r = r[1:-1, 1:-1, 1:-1]
    eig = [scipy.linalg.eigh(K1[a][1:-1, 1:-1], M1[a][1:-1, 1:-1]) for a in range(3)]
    (l0, V0), (l1, V1), (l2, V2) = eig
    rh = tables.kron_apply(V0.T, V1.T, V2.T, r)
    rh /= l0[:, None, None] + l1[None, :, None] + l2[None, None, :]
    H = Hb.copy()
    H[1:-1, 1:-1, 1:-1] = tables.kron_apply(V0, V1, V2, rh)
    return H, tuple(x1)


@functools.lru_cache(maxsize=64)
def fine_type_table(p, q, t3, half_width, refine, ngl=6, nodes=NODES):
    """The potential of the type-t3 basis screen on its box (as type_table) from an
    order-p Galerkin solve on a mesh refine times finer (element size 1 / refine):
    the stand-in for the continuum potential of Eq. sc (FE error ~ refine^-(p+1) of
    the table's).  H[ix, iy, iz] at x = lo + k / (p refine)."""
    ext = [box_extent(t, half_width) for t in t3]
    nel = [refine * (hi - lo) for (lo, hi) in ext]
    hf = 1.0 / refine
    Me, Ke = fe1d.element_matrices(p, hf)
    M1 = [fe1d.assemble_open(Me, ne, p) for ne in nel]
    K1 = [fe1d.assemble_open(Ke, ne, p) for ne in nel]
    tq, wq = fe1d.gauss_legendre01(p + q + 2)
    m1 = []
    for t, (lo, _), ne in zip(t3, ext, nel):
        col = np.zeros(p * ne + 1)
        for e in range(ne):
            x = lo + (e + tq) * hf
            psi = np.zeros_like(x)
            for (a, b, f) in basis_pieces_1d(q, t, nodes):
                inside = (x >= a) & (x <= b)
                psi = np.where(inside, f(np.clip(x, a, b)), psi)
            col[p * e:p * e + p + 1] += hf * np.einsum('g,g,gk->k', wq, psi, fe1d.lagrange_values(p, tq))
        m1.append(col)
    rhs = 4.0 * np.pi * m1[0][:, None, None] * m1[1][None, :, None] * m1[2][None, None, :]
    x1 = [lo + np.arange(p * ne + 1) * (hf / p) for (lo, _), ne in zip(ext, nel)]
    N = [len(x) for x in x1]
    I, J, K = np.meshgrid(np.arange(N[0]), np.arange(N[1]), np.arange(N[2]), indexing='ij')
    onb = (I == 0) | (I == N[0] - 1) | (J == 0) | (J == N[1] - 1) | (K == 0) | (K == N[2] - 1)
    Hb = np.zeros(tuple(N))
    pts = np.stack([x1[0][I[onb]], x1[1][J[onb]], x1[2][K[onb]]], axis=1)
    Hb[onb] = basis_potential_continuum(q, t3, pts, ngl, nodes)
    r = rhs - (tables.kron_apply(K1[0], M1[1], M1[2], Hb) + tables.kron_apply(M1[0], K1[1], M1[2], Hb)
               + tables.kron_apply(M1[0], M1[1], K1[2], Hb))
    r = r[1:-1, 1:-1, 1:-1]
    eig = [scipy.linalg.eigh(K1[a][1:-1, 1:-1], M1[a][1:-1, 1:-1]) for a in range(3)]
    (l0, V0), (l1, V1), (l2, V2) = eig
    rh = tables.kron_apply(V0.T, V1.T, V2.T, r)
    rh /= l0[:, None, None] + l1[None, :, None] + l2[None, None, :]
    H = Hb.copy()
    H[1:-1, 1:-1, 1:-1] = tables.kron_apply(V0, V1, V2, rh)
    return H, tuple(x1)


def evaluate_fine_table(H, x1, p, refine, pts):
    """The fine table at points (M, 3) (anchor-relative, element units) with the order-p
    basis of the fine element holding each point."""
    lo = np.array([x[0] for x in x1])
    u = (pts - lo) * refine                                  # fine-element units
    nfe = np.array([(len(x) - 1) // p for x in x1])
    e = np.clip(np.floor(u).astype(np.int64), 0, nfe - 1)
    t = u - e
    lv = [fe1d.lagrange_values(p, t[:, a]) for a in range(3)]
    out = np.zeros(len(pts))
    for mx in range(p + 1):
        for my in range(p + 1):
            for mz in range(p + 1):
                out += (H[p * e[:, 0] + mx, p * e[:, 1] + my, p * e[:, 2] + mz]
                        * lv[0][:, mx] * lv[1][:, my] * lv[2][:, mz])
    return out


def kept_tables(p, q, keep, half_width=None, ngl=6, interior_only=False, nodes=NODES):
    """Nodal values of each type's table on [-keep, keep]^3 about its anchor:
    dict t3 -> array ((2 keep p + 1),)*3; interior_only: the types with no vertex
    factor (all that one-element screens use)."""
    if half_width is None:
        half_width = keep + 2
    out = {}
    for t3 in itertools.product(range(1 if interior_only else 0, q), repeat=3):
        H, _ = type_table(p, q, t3, half_width, ngl, nodes)
        s = p * (half_width - keep)
        e = p * (half_width + keep) + 1
        out[t3] = H[s:e, s:e, s:e]
    return out


def local_node(kappa, q):
    """kappa = i + (q+1) j + (q+1)^2 k -> (i, j, k)."""
    q1 = q + 1
    return np.array([kappa % q1, (kappa // q1) % q1, kappa // (q1 * q1)])


def one_element_coefficients(q, h, delta3, nodes=NODES):
    """Screens confined to the charge's element (one-element screens, Sec. 5.3): only the
    (q-1)^3 interior nodes carry weight.  Per axis the q - 1 interior weights solve the
    moment system of Eq. moment1d for l = 0 .. q-2 (the interior functions vanish outside
    the element, so their moments are the rows l < q - 1, columns 1 .. q-1 of the
    patch moment matrix).  Returns (..., (q+1)^3), zero on the element's face nodes."""
    assert q >= 2, "a one-element screen needs an interior node"
    delta3 = np.asarray(delta3, dtype=np.float64)
    Om = screens.moment_matrix_1d(q, h, nodes)[:q - 1, 1:q]
    w = []
    for a in range(3):
        rhs = np.stack([delta3[..., a] ** l for l in range(q - 1)], axis=-1)
        wi = np.linalg.solve(Om, rhs[..., None])[..., 0]
        full = np.zeros(delta3.shape[:-1] + (q + 1,))
        full[..., 1:q] = wi
        w.append(full)
    c = w[2][..., :, None, None] * w[1][..., None, :, None] * w[0][..., None, None, :]
    return c.reshape(delta3.shape[:-1] + ((q + 1) ** 3,))


def element_coefficients(bins, Q, n, q, support='patch', nodes=NODES):
    """C[e, kappa] = sum_{j in e} Q_j c_kappa(delta_j), shape (n^3, (q+1)^3), units charge/h^3.
    support='patch': the screens of Eq. moment1d on the element's (q+1)^3 nodes;
    support='element': one-element screens on its interior nodes."""
    if support == 'element':
        c = one_element_coefficients(q, bins['h'], bins['delta'], nodes)
    else:
        c = screens.screen_coefficients(q, bins['h'], bins['delta'], nodes)
    C = np.zeros((n ** 3, c.shape[1]))
    np.add.at(C, bins['cell'], np.asarray(Q)[:, None] * c)
    return C


def nodal_density(C, n, q):
    """Order-q nodal screen density on the periodic order-q mesh (Eq. assign): element
    (ex, ey, ez)'s local node (i, j, k) is the global node (q ex + i, q ey + j, q ez + k)
    mod q n.  Returns r indexed [ix, iy, iz]."""
    q1, N = q + 1, q * n
    Cg = C.reshape(n, n, n, q1, q1, q1)        # [ez, ey, ex, k, j, i]
    r = np.zeros((N, N, N))
    e = np.arange(n)
    for i, j, k in itertools.product(range(q1), repeat=3):
        contrib = np.transpose(Cg[:, :, :, k, j, i], (2, 1, 0))   # [ex, ey, ez]
        r[np.ix_((q * e + i) % N, (q * e + j) % N, (q * e + k) % N)] += contrib
    return r


def screen_window_matrix(n_sr, p, q, kept):
    """W[(d, kappa), m]: nodal value, at node m of the target element, of the table of
    local node kappa of the source element at offset d from the target.  Along an axis
    the node's anchor is the source element's left vertex plus s (s = 1 for local
    index q), so target node m sits at -d - s + m / p from it; the kept tables start
    at -keep with step 1 / p."""
    keep = n_sr + 1
    offs = block_offsets(n_sr)
    p1, q1 = p + 1, q + 1
    m = np.arange(p1 ** 3)
    mm = np.stack([m % p1, (m // p1) % p1, m // (p1 * p1)], axis=1)
    W = np.zeros((len(offs), q1 ** 3, p1 ** 3))
    for kap in range(q1 ** 3):
        loc = local_node(kap, q)
        s = (loc == q).astype(int)
        t3 = tuple(int(x) for x in loc % q)
        if t3 not in kept:
            continue                              # a node no screen uses (one-element screens)
        Hk = kept[t3]
        for k, d in enumerate(offs):
            base = p * (-d - s + keep)
            W[k, kap] = Hk[base[0] + mm[:, 0], base[1] + mm[:, 1], base[2] + mm[:, 2]]
    return W.reshape(len(offs) * q1 ** 3, p1 ** 3)


def forward(pos, Q, L, n, q, n_sr=3, neutralise=True, chunk=1024, half_width=None, ngl=6, support='patch',
            nodes=NODES, screen_tables='fe', refine=3):
    """Phi_i and U for charges Q at pos (N x 3) with order-q screens and the order p = q + 2
    mesh (Sec. 2: p = q + 2), with the intermediates.  support='element' uses one-element
    screens (Sec. 5.3), still with p = q + 2.  nodes: the node set of the order-q screen
    basis ('gll' or 'equispaced'); the order-p mesh space does not depend on it.
    screen_tables='fe': the screen potentials through the FE tables, evaluated with the
    target element's order-p basis (the Remark of Sec. 4); 'continuum': through the
    tables of a refine-times finer mesh evaluated at the charge itself, standing in for
    the continuum tables of Eq. sc."""
    pos = np.asarray(pos, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    assert n >= 2 * n_sr + 1, "the short-range block must not wrap onto itself"
    p = q + 2
    bins = bin_particles(pos, L, n)
    h = bins['h']
    C = element_coefficients(bins, Q, n, q, support, nodes)
    r = nodal_density(C, n, q)
    ops = MeshOperators(L, n, p, q, nodes)
    b = ops.load_vector(r)
    if neutralise:
        b = ops.neutralise(b)
    phi_mesh = ops.solve(b)
    U3, _ = q3_basis(bins, p)
    ix, iy, iz = element_node_index(bins['c3'], n, p)
    phi_sm = np.einsum('nm,nm->n', phi_mesh[ix, iy, iz], U3)
    phi_sing, _ = singular_sums(bins, Q, n, n_sr)
    kept = kept_tables(p, q, n_sr + 1, half_width, ngl, interior_only=support == 'element', nodes=nodes)
    Wmat = screen_window_matrix(n_sr, p, q, kept)
    offs = block_offsets(n_sr)
    phi_scr = np.zeros(len(Q))
    for s0 in range(0, len(Q), chunk):
        sl = slice(s0, s0 + chunk)
        Cblk = gather_block_coefficients(C, bins['c3'][sl], n, offs)
        phi_scr[sl] = np.einsum('nm,nm->n', (h * h) * (Cblk @ Wmat), U3[sl])
    if screen_tables == 'continuum':
        phi_scr = continuum_screen_part(bins, C, n, q, p, n_sr, half_width, refine, ngl, nodes)
    phi = phi_sm + phi_sing - phi_scr
    return dict(phi=phi, U=0.5 * np.dot(Q, phi), phi_sm=phi_sm, phi_sing=phi_sing, phi_scr=phi_scr,
                phi_mesh=phi_mesh, r=r, b=b, C=C, bins=bins, ops=ops, Wmat=Wmat, p=p, q=q)


def continuum_screen_part(bins, C, n, q, p, n_sr, half_width, refine, ngl, nodes):
    """Screen potentials of the block's charges at each charge from the fine tables,
    evaluated at the charge's own position (Eq. sc form)."""
    keep = n_sr + 1
    hw = keep + 2 if half_width is None else half_width
    h = bins['h']
    c3, delta = bins['c3'], bins['delta']
    tables_f = {t3: fine_type_table(p, q, t3, hw, refine, ngl, nodes) for t3 in itertools.product(range(q), repeat=3)}
    x_loc = delta / h + 0.5                                   # target position in its element, element units
    out = np.zeros(len(c3))
    for d in block_offsets(n_sr):
        src = (c3 + d) % n
        s = src[:, 0] + n * src[:, 1] + n * n * src[:, 2]
        for kap in range((q + 1) ** 3):
            w = C[s, kap]
            if not np.any(w):
                continue
            loc = local_node(kap, q)
            anchor = d + (loc == q)                           # anchor vertex, target element units
            H, x1 = tables_f[tuple(int(v) for v in loc % q)]
            out += (h * h) * w * evaluate_fine_table(H, x1, p, refine, x_loc - anchor)
    return out
