"""The 1-D eigenbasis behind the fast-diagonalisation mesh solve, built on the host from the block-circulant
structure of the periodic order-3 matrices (one small problem per wavenumber), against a dense generalized
eigensolver on the oracle's matrices (whose element integrals are pinned by exact rational integration).
Host code only: runs without a GPU."""
import ctypes

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import fe1d


@pytest.fixture(scope="module")
def lib():
    from paper_1503_08509_gb300 import _lib, build
    build.build()
    return _lib.load()


def eigenbasis(lib, n):
    N = 3 * n
    lam = np.empty(N)
    V = np.empty((N, N))
    st = lib.fep3m_mesh_eigenbasis(n, lam.ctypes.data_as(ctypes.c_void_p), V.ctypes.data_as(ctypes.c_void_p))
    assert st == 0
    return lam, V


def dense(a):
    return np.asarray(a.todense()) if hasattr(a, "todense") else np.asarray(a)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33])
def test_eigenbasis_matches_dense_solver(lib, n):
    lam, V = eigenbasis(lib, n)
    M1, K1, _ = fe1d.periodic_matrices(3, n, 1.0, 1)
    M1, K1 = dense(M1), dense(K1)
    ref = sl.eigh(K1, M1, eigvals_only=True)
    scale = np.abs(ref).max()
    assert np.abs(np.sort(lam) - ref).max() < 1e-11 * scale
    N = 3 * n
    assert np.abs(V.T @ M1 @ V - np.eye(N)).max() < 1e-12
    assert np.abs(K1 @ V - M1 @ V * lam[None, :]).max() < 1e-11 * scale
    # exactly one constant mode with eigenvalue zero
    null = np.argmin(np.abs(lam))
    assert abs(lam[null]) < 1e-12 * scale
    assert np.ptp(V[:, null]) < 1e-12


def test_eigenbasis_rejects_bad_sizes(lib):
    lam = np.empty(3)
    V = np.empty((3, 3))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.fep3m_mesh_eigenbasis(0, p(lam), p(V)) != 0
    assert lib.fep3m_mesh_eigenbasis(5000, p(lam), p(V)) != 0
