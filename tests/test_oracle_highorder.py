"""Pins for the order-q screen oracle (oracle.highorder): screens of order q >= 2 with the
order p = q + 2 mesh (Sec. 2.1, Sec. 2.4, the Remark of Sec. 4, Fig. decayavg, Fig. compareerr)."""
import itertools

import numpy as np
import pytest

from oracle import ewald, fe1d, fep3m, highorder, screens, tables
from paper_1503_08509_gb300 import workloads


def test_q1_table_is_the_hat_table():
    # for q = 1 the only basis-screen type is the vertex hat of oracle.tables
    H, _ = tables.basis_screen_table(3, 8, 8)
    H1, _ = highorder.type_table(3, 1, (0, 0, 0), 8, 8)
    assert np.abs(H - H1).max() < 1e-14 * np.abs(H).max()


def test_q1_reduces_to_the_q1_oracle():
    pos, Q = workloads.uniform_pm(60, seed=6)
    a = fep3m.forward(pos, Q, 1.0, 8)
    b = highorder.forward(pos, Q, 1.0, 8, 1, half_width=8, ngl=8)
    assert np.abs(a['phi'] - b['phi']).max() < 1e-13 * np.abs(a['phi']).max()


@pytest.mark.parametrize("q", [2, 3])
def test_type_tables_symmetries(q):
    # every box is symmetric about its screen's support: type 0 is even about its
    # vertex, interior type i is the mirror image of type q - i about the element
    # centre, and permuting the axes permutes the types
    p, hw = q + 2, 3
    T = {t3: highorder.type_table(p, q, t3, hw, 6)[0] for t3 in itertools.product(range(q), repeat=3)}
    scale = max(np.abs(H).max() for H in T.values())
    for t3, H in T.items():
        for perm in itertools.permutations(range(3)):
            tp = tuple(t3[a] for a in perm)
            assert np.abs(T[tp] - H.transpose(perm)).max() < 1e-12 * scale, (t3, perm)
        for a in range(3):
            tm = list(t3)
            tm[a] = (q - t3[a]) % q
            assert np.abs(T[tuple(tm)] - np.flip(H, axis=a)).max() < 1e-12 * scale, (t3, a)


def independent_mixed_column(p, q, node, lo, nel):
    """int phi^p_k psi dx with psi the order-q nodal function of the centred element's
    local node `node` (oracle.screens.omega_pieces, element [-1/2, 1/2]), shifted so its
    anchor vertex sits at 0, by Gauss-Legendre quadrature of the product on each element."""
    pieces = screens.omega_pieces(q, 1.0, highorder.NODES)[node]
    shift = 0.5 - (1.0 if node == q else 0.0)
    t, w = fe1d.gauss_legendre01(p + q + 2)
    m1 = np.zeros(p * nel + 1)
    for e in range(nel):
        x = lo + e + t
        psi = np.zeros_like(x)
        for (a, b, f) in pieces:
            inside = (x - shift >= a) & (x - shift <= b)
            psi = np.where(inside, f(np.clip(x - shift, a, b)), psi)
        m1[p * e:p * e + p + 1] += np.einsum('g,g,gk->k', w, psi, fe1d.lagrange_values(p, t))
    return m1


@pytest.mark.parametrize("q, t3", [(2, (0, 0, 0)), (2, (1, 0, 1)), (3, (2, 0, 1)), (3, (0, 1, 2))])
def test_type_table_solves_dirichlet_problem(q, t3):
    p, hw = q + 2, 3
    H, x1 = highorder.type_table(p, q, t3, hw, 6)
    ext = [highorder.box_extent(t, hw) for t in t3]
    nel = [hi - lo for lo, hi in ext]
    Me, Ke = fe1d.element_matrices(p, 1.0)
    M1 = [fe1d.assemble_open(Me, ne, p) for ne in nel]
    K1 = [fe1d.assemble_open(Ke, ne, p) for ne in nel]
    m1 = [independent_mixed_column(p, q, t, lo, ne) for t, (lo, _), ne in zip(t3, ext, nel)]
    rhs = 4 * np.pi * m1[0][:, None, None] * m1[1][None, :, None] * m1[2][None, None, :]
    KH = (tables.kron_apply(K1[0], M1[1], M1[2], H) + tables.kron_apply(M1[0], K1[1], M1[2], H)
          + tables.kron_apply(M1[0], M1[1], K1[2], H))
    assert np.abs((KH - rhs)[1:-1, 1:-1, 1:-1]).max() < 1e-12 * np.abs(rhs).max()
    # boundary rows: the continuum potential, here with a finer quadrature
    pts = np.array([[x1[0][0], x1[1][3], x1[2][7]], [x1[0][-1], x1[1][-1], x1[2][9]]])
    ref = highorder.basis_potential_continuum(q, t3, pts, ngl=16)
    assert np.allclose([H[0, 3, 7], H[-1, -1, 9]], ref, rtol=1e-11, atol=0)


def screen_node_integrals(q, n, h):
    """Integrals of the periodic order-q screen basis functions (the oracle's node set)."""
    t, wg = fe1d.gauss_legendre01(q + 2)
    we = h * np.einsum('g,gi->i', wg, fe1d.lagrange_values(q, t, highorder.NODES))
    out = np.zeros(q * n)
    for e in range(n):
        for i in range(q + 1):
            out[(q * e + i) % (q * n)] += we[i]
    return out


@pytest.mark.parametrize("q", [2, 3])
def test_nodal_density_carries_charge_and_dipole(q):
    # Eq. moment1d with l = 0, 1: the screens hold each charge's total and its first
    # moments, so the order-q nodal density integrates to sum Q and sum Q x
    n, L = 5, 1.0
    pos, Q = workloads.uniform_pm(40, seed=4)
    pos = pos * 0.6 + 0.2                             # away from the periodic seam
    b = fep3m.bin_particles(pos, L, n)
    r = highorder.nodal_density(highorder.element_coefficients(b, Q, n, q), n, q)
    w = screen_node_integrals(q, n, L / n)
    assert abs(np.einsum('ijk,i,j,k->', r, w, w, w) - Q.sum()) < 1e-12 * np.abs(Q).sum()
    # first moment along x: nodes of the order-q mesh at i h / q, integrated with
    # x * psi_i (the density's support crosses no periodic seam here)
    t, wg = fe1d.gauss_legendre01(q + 2)
    h = L / n
    wx = np.zeros(q * n)
    for e in range(n):
        x = (e + t) * h
        lv = fe1d.lagrange_values(q, t, highorder.NODES)
        for i in range(q + 1):
            wx[(q * e + i) % (q * n)] += h * np.sum(wg * x * lv[:, i])
    mx = np.einsum('ijk,i,j,k->', r, wx, w, w)
    assert abs(mx - np.dot(Q, pos[:, 0])) < 1e-12 * np.abs(Q).sum()


@pytest.mark.parametrize("q", [2, 3])
def test_screened_potential_decays_like_r_minus_q_plus_2(q):
    # Fig. decayavg: the charge-plus-screen potential of order q decays like R^-(q+2);
    # the screen is built from the type/anchor map the tables use (local node i of
    # the element [-1/2, 1/2]: anchor -1/2 + [i = q], type i mod q)
    delta = np.array([0.23, -0.11, 0.37])
    c = screens.screen_coefficients(q, 1.0, delta[None, :], highorder.NODES)[0]
    rng = np.random.default_rng(1)
    dirs = rng.normal(size=(16, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    vals = {}
    for R in (4.0, 8.0):
        x = delta + R * dirs
        phi_sc = np.zeros(len(x))
        for kap in range((q + 1) ** 3):
            loc = highorder.local_node(kap, q)
            anchor = -0.5 + (loc == q)
            t3 = tuple(int(v) for v in loc % q)
            phi_sc += c[kap] * highorder.basis_potential_continuum(q, t3, x - anchor, ngl=12)
        vals[R] = np.sqrt(np.mean((1.0 / R - phi_sc) ** 2))
    slope = np.log(vals[8.0] / vals[4.0]) / np.log(2.0)
    assert -(q + 2) - 0.35 < slope < -(q + 2) + 0.35, slope


def test_whole_element_shift_is_exact_q2():
    pos, Q = workloads.uniform_pm(50, seed=12)
    n = 7
    a = highorder.forward(pos, Q, 1.0, n, 2, n_sr=2)
    b = highorder.forward(pos + np.array([1, -2, 3]) / n, Q, 1.0, n, 2, n_sr=2)
    assert np.abs(a['phi'] - b['phi']).max() < 1e-11 * np.abs(a['phi']).max()


def test_error_against_ewald_falls_with_q():
    # Fig. compareerr: the error against a converged Ewald sum falls fast with q
    # (measured here: 8.0e-3, 1.6e-3, 2.1e-4 for q = 1, 2, 3 at n = 8, n_sr = 2)
    pos, Q = workloads.uniform_pm(100, seed=9)
    pe = ewald.ewald(pos, Q, 1.0)
    err = {}
    for q in (1, 2, 3):
        d = highorder.forward(pos, Q, 1.0, 8, q, n_sr=2)['phi'] - pe
        d -= d.mean()                                   # potentials agree up to a constant (Sec. 4)
        err[q] = np.linalg.norm(d) / np.linalg.norm(pe)
    assert err[1] < 2e-2, err
    assert err[2] < err[1] / 3 and err[3] < err[2] / 3, err


# ------------------------------------------------- one-element screens (Sec. 5.3)
def one_element_screened_rms(q, Rs):
    delta = np.array([0.21, -0.1, 0.33])
    c = highorder.one_element_coefficients(q, 1.0, delta[None, :])[0]
    rng = np.random.default_rng(1)
    dirs = rng.normal(size=(16, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    out = {}
    for R in Rs:
        x = delta + R * dirs
        phi = np.zeros(len(x))
        for kap in np.flatnonzero(c):
            loc = highorder.local_node(kap, q)
            assert np.all((loc > 0) & (loc < q))             # interior nodes only
            phi += c[kap] * highorder.basis_potential_continuum(q, tuple(int(v) for v in loc), x + 0.5, ngl=12)
        out[R] = np.sqrt(np.mean((1.0 / R - phi) ** 2))
    return out


@pytest.mark.parametrize("q", [2, 3, 4])
def test_one_element_screens_decay_like_r_minus_q(q):
    # Sec. 5.3: confining the screen to the charge's element loses two powers of decay
    # (q = 3 gives R^-3 instead of R^-5), but the asymptotic rate starts near R^ = 1
    # instead of 3: the slope is already -q between 2 and 4 element widths
    v = one_element_screened_rms(q, (2.0, 4.0, 8.0))
    far = np.log(v[8.0] / v[4.0]) / np.log(2.0)
    near = np.log(v[4.0] / v[2.0]) / np.log(2.0)
    assert abs(far + q) < 0.15 and abs(near + q) < 0.2, (far, near)


def test_one_element_density_stays_in_the_element_and_keeps_charge_and_dipole():
    q, n, L = 3, 5, 1.0
    pos, Q = workloads.uniform_pm(40, seed=4)
    pos = pos * 0.6 + 0.2
    b = fep3m.bin_particles(pos, L, n)
    r = highorder.nodal_density(highorder.element_coefficients(b, Q, n, q, 'element'), n, q)
    idx = np.arange(q * n)
    face = (idx % q) == 0
    assert np.all(r[face, :, :] == 0) and np.all(r[:, face, :] == 0) and np.all(r[:, :, face] == 0)
    w = screen_node_integrals(q, n, L / n)
    assert abs(np.einsum('ijk,i,j,k->', r, w, w, w) - Q.sum()) < 1e-12 * np.abs(Q).sum()
    h = L / n
    t, wg = fe1d.gauss_legendre01(q + 2)
    wx = np.zeros(q * n)
    for e in range(n):
        lv = fe1d.lagrange_values(q, t, highorder.NODES)
        for i in range(q + 1):
            wx[(q * e + i) % (q * n)] += h * np.sum(wg * (e + t) * h * lv[:, i])
    assert abs(np.einsum('ijk,i,j,k->', r, w, wx, w) - np.dot(Q, pos[:, 1])) < 1e-12 * np.abs(Q).sum()


def test_one_element_screens_against_ewald():
    # measured: 7.4e-3 (q = 3) and 3.9e-4 (q = 4) at n = 8, n_sr = 2
    pos, Q = workloads.uniform_pm(100, seed=9)
    pe = ewald.ewald(pos, Q, 1.0)
    err = {}
    for q in (3, 4):
        d = highorder.forward(pos, Q, 1.0, 8, q, n_sr=2, support='element')['phi'] - pe
        d -= d.mean()
        err[q] = np.linalg.norm(d) / np.linalg.norm(pe)
    assert err[3] < 2e-2 and err[4] < err[3] / 5, err


# ------------------------------------------------------ node set of the screen basis
@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_gauss_lobatto_nodes(q):
    # the Gauss-Lobatto rule on these nodes (weights = integrals of the Lagrange basis)
    # integrates polynomials of degree 2q - 1 exactly; q <= 2 gives the equispaced set
    x = fe1d.gll_nodes01(q)
    t, wg = fe1d.gauss_legendre01(q + 2)
    w = np.einsum('g,gi->i', wg, fe1d.lagrange_values(q, t, 'gll'))
    for k in range(2 * q):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14, k
    if q <= 2:
        assert np.array_equal(x, np.linspace(0.0, 1.0, q + 1))


def test_error_on_the_paper_workload_falls_faster_with_each_q():
    # Sec. 4 / Fig. compareerr: two biased cubes, h = 1/15, 7^3 block, q = 1 .. 4;
    # measured 2.9e-3, 3.2e-4, 2.3e-5, 1.5e-6: each step of q gains more than the last
    pos, Q = workloads.two_biased_cubes(120)
    pe = ewald.ewald(pos, Q, 1.0)
    err = []
    for q in (1, 2, 3, 4):
        d = highorder.forward(pos, Q, 1.0, 15, q, n_sr=3)['phi'] - pe
        d -= d.mean()
        err.append(np.linalg.norm(d) / np.linalg.norm(pe))
    gain = [err[i] / err[i + 1] for i in range(3)]
    assert err[0] < 5e-3 and gain[0] > 5 and gain[1] > gain[0] and gain[2] > gain[1], (err, gain)


# ------------------------------------- continuum tables (Eq. sc) against the FE form
@pytest.mark.parametrize("t3", [(0, 0, 0), (1, 0, 1)])
def test_fine_tables_approach_the_continuum(t3):
    # the stand-in for the continuum tables: refined FE solutions, which agree with the
    # continuum potential away from the screen and converge under refinement near it
    q, p, hw = 2, 4, 3
    H3, x3 = highorder.fine_type_table(p, q, t3, hw, 3)
    H4, x4 = highorder.fine_type_table(p, q, t3, hw, 4)
    rng = np.random.default_rng(0)
    near = rng.uniform(-1.5, 2.0, size=(200, 3))
    far = rng.uniform(-3, 3, size=(3000, 3))
    far = far[np.linalg.norm(far - 0.5, axis=1) > 2.5][:100]
    a = highorder.evaluate_fine_table(H3, x3, p, 3, near)
    b = highorder.evaluate_fine_table(H4, x4, p, 4, near)
    assert np.abs(a - b).max() < 2e-4 * np.abs(b).max()
    c = highorder.basis_potential_continuum(q, t3, far, ngl=10)
    assert np.abs(highorder.evaluate_fine_table(H3, x3, p, 3, far) - c).max() < 1e-6 * np.abs(c).max()


def test_fe_form_of_the_tables_beats_the_continuum_form_at_q2():
    # the Remark of Sec. 4 stores the tables as order-p FE solutions evaluated like the
    # mesh potential; against screen potentials evaluated at the charges (Eq. sc) that
    # keeps the FE error of the nearby screens inside the one FE space, where it cancels
    # against the mesh part: measured 1.6e-3 against 1.0e-2 (q = 2, n = 8, n_sr = 2)
    pos, Q = workloads.uniform_pm(100, seed=9)
    pe = ewald.ewald(pos, Q, 1.0)
    err = {}
    for form in ('fe', 'continuum'):
        d = highorder.forward(pos, Q, 1.0, 8, 2, n_sr=2, screen_tables=form)['phi'] - pe
        d -= d.mean()
        err[form] = np.linalg.norm(d) / np.linalg.norm(pe)
    assert err['fe'] < err['continuum'] / 3, err
