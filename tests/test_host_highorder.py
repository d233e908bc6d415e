"""Host-only building blocks for screens of order q >= 2 (C ABI, no GPU): the periodic
order-p eigenbasis against a dense generalized eigensolver on the oracle's matrices, and
the basis-screen type tables against the oracle's (oracle.highorder)."""
import ctypes

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import fe1d, highorder, tables


@pytest.fixture(scope="module")
def lib():
    from paper_1503_08509_gb300 import _lib, build
    build.build()
    return _lib.load()


def ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [1, 2, 3, 8])
def test_order_p_eigenbasis_matches_dense_solver(lib, p, n):
    N = p * n
    lam, V = np.empty(N), np.empty((N, N))
    assert lib.fep3m_mesh_eigenbasis_order(p, n, ptr(lam), ptr(V)) == 0
    M1, K1, _ = fe1d.periodic_matrices(p, n, 1.0, 1)
    ref = sl.eigh(K1, M1, eigvals_only=True)
    scale = max(np.abs(ref).max(), 1.0)                  # p = n = 1: the single eigenvalue is 0
    assert np.abs(np.sort(lam) - ref).max() < 1e-11 * scale
    assert np.abs(V.T @ M1 @ V - np.eye(N)).max() < 1e-11
    assert np.abs(V.T @ K1 @ V - np.diag(lam)).max() < 1e-11 * scale


def test_order_3_eigenbasis_is_the_mesh_solver_basis(lib):
    n = 7
    a, Va, b, Vb = np.empty(21), np.empty((21, 21)), np.empty(21), np.empty((21, 21))
    assert lib.fep3m_mesh_eigenbasis_order(3, n, ptr(a), ptr(Va)) == 0
    assert lib.fep3m_mesh_eigenbasis(n, ptr(b), ptr(Vb)) == 0
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def type_table(lib, q, t3, n_sr, pad):
    K = 2 * (n_sr + 1) * (q + 2) + 1
    out = np.empty(K ** 3)
    assert lib.fep3m_screen_type_table(q, t3[0], t3[1], t3[2], n_sr, pad, ptr(out)) == 0
    return out.reshape(K, K, K).transpose(2, 1, 0)        # [ix, iy, iz]


def test_q1_type_table_is_the_hat_table(lib):
    n_sr, pad = 1, 2
    ref = tables.kept_table(3, half_width=n_sr + 1 + pad, ngl=8, keep=n_sr + 1)
    assert np.abs(type_table(lib, 1, (0, 0, 0), n_sr, pad) - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("q, t3", [(2, (0, 0, 0)), (2, (1, 0, 0)), (2, (0, 1, 1)), (3, (2, 1, 0)), (3, (1, 1, 1))])
def test_type_tables_match_the_oracle(lib, q, t3):
    n_sr, pad = 1, 1
    keep = n_sr + 1
    H, _ = highorder.type_table(q + 2, q, t3, keep + pad, 8)
    s = (q + 2) * pad
    ref = H[s:H.shape[0] - s - (q + 2) * (t3[0] > 0), s:H.shape[1] - s - (q + 2) * (t3[1] > 0),
            s:H.shape[2] - s - (q + 2) * (t3[2] > 0)]
    got = type_table(lib, q, t3, n_sr, pad)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_bad_arguments_are_rejected(lib):
    out = np.empty(1)
    assert lib.fep3m_mesh_eigenbasis_order(0, 4, ptr(out), ptr(out)) != 0
    assert lib.fep3m_mesh_eigenbasis_order(9, 4, ptr(out), ptr(out)) != 0
    assert lib.fep3m_screen_type_table(2, 2, 0, 0, 1, 1, ptr(out)) != 0     # type out of range
    assert lib.fep3m_screen_type_table(5, 0, 0, 0, 1, 1, ptr(out)) != 0     # q out of range
    assert lib.fep3m_screen_type_table(2, 0, 0, 0, 0, 1, ptr(out)) != 0     # n_sr out of range


@pytest.mark.parametrize("q, n_sr", [(1, 2), (2, 1), (3, 1)])
def test_node_table_regroups_the_window_contraction(lib, q, n_sr):
    # the block's screens at a target element's nodes, regrouped by screen node u,
    # equal the oracle's per-source-element window contraction
    from oracle import fep3m
    p, keep, pad = q + 2, n_sr + 1, 1
    U, M = (2 * n_sr + 1) * q + 1, (p + 1) ** 3
    H = np.empty(U ** 3 * M)
    assert lib.fep3m_screen_node_table(q, n_sr, pad, ptr(H)) == 0
    H = H.reshape(U ** 3, M)
    n = 2 * n_sr + 3
    rng = np.random.default_rng(q)
    C = rng.normal(size=(n ** 3, (q + 1) ** 3))
    c3 = rng.integers(0, n, size=(6, 3))
    offs = fep3m.block_offsets(n_sr)
    kept = highorder.kept_tables(p, q, keep, half_width=keep + pad, ngl=8)
    ref = fep3m.gather_block_coefficients(C, c3, n, offs) @ highorder.screen_window_matrix(n_sr, p, q, kept)
    A = np.zeros((len(c3), U ** 3))
    for t, e in enumerate(c3):
        for d in offs:
            s = (e + d) % n
            for kap in range((q + 1) ** 3):
                o = q * keep - (q * d + highorder.local_node(kap, q))
                A[t, o[0] + U * (o[1] + U * o[2])] += C[s[0] + n * s[1] + n * n * s[2], kap]
    got = A @ H
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    if q == 1:
        # the order-1 vertex-offset layout: row o reads the hat table at 3 o + m
        K = 6 * keep + 1
        T = np.empty(K ** 3)
        assert lib.fep3m_screen_type_table(1, 0, 0, 0, n_sr, pad, ptr(T)) == 0
        T = T.reshape(K, K, K)                           # [z][y][x]
        o, m = (1, 4, 2), (3, 0, 2)
        row = o[0] + U * (o[1] + U * o[2])
        assert H[row, m[0] + 4 * (m[1] + 4 * m[2])] == T[3 * o[2] + m[2], 3 * o[1] + m[1], 3 * o[0] + m[0]]


@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("one_element", [False, True])
def test_screen_weight_polynomials_match_the_oracle(lib, q, one_element):
    if one_element and q < 2:
        return
    W = np.empty((q + 1) ** 2)
    assert lib.fep3m_screen_weight_poly(q, int(one_element), ptr(W)) == 0
    W = W.reshape(q + 1, q + 1)                        # [node i][power l]
    h = 0.37
    delta = np.linspace(-0.5, 0.5, 7) * h
    got = np.stack([np.polyval(W[i][::-1], delta / h) / h for i in range(q + 1)], axis=-1)
    from oracle import screens
    if one_element:
        # the oracle's one-element system: interior functions, moments l < q - 1
        Om = screens.moment_matrix_1d(q, h, highorder.NODES)[:q - 1, 1:q]
        rhs = np.stack([delta ** l for l in range(q - 1)], axis=0)
        ref = np.linalg.solve(Om, rhs).T
        assert np.allclose(got[:, 1:q], ref, rtol=1e-11, atol=1e-11 / h)
        assert np.all(got[:, 0] == 0) and np.all(got[:, q] == 0)
    else:
        ref = screens.screen_weights_1d(q, h, delta, highorder.NODES)
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 / h)


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("n", [1, 4, 9])
@pytest.mark.parametrize("dirichlet", [True, False])
def test_box_eigenbasis_matches_dense_solver(lib, p, n, dirichlet):
    if dirichlet and p * n < 2:
        return
    Me, Ke = fe1d.element_matrices(p, 1.0)
    M1, K1 = fe1d.assemble_open(Me, n, p), fe1d.assemble_open(Ke, n, p)
    if dirichlet:
        M1, K1 = M1[1:-1, 1:-1], K1[1:-1, 1:-1]
    N = len(M1)
    lam, V = np.empty(N), np.empty((N, N))
    assert lib.fep3m_box_eigenbasis(p, n, int(dirichlet), ptr(lam), ptr(V)) == 0
    ref = sl.eigh(K1, M1, eigvals_only=True)
    scale = max(np.abs(ref).max(), 1.0)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(lam - ref).max() < 1e-10 * scale
    assert np.abs(V.T @ M1 @ V - np.eye(N)).max() < 1e-10
    assert np.abs(V.T @ K1 @ V - np.diag(lam)).max() < 1e-10 * scale
    if not dirichlet:
        assert abs(lam[0]) < 1e-10 * scale                # the constant mode
