"""Pins for the Neumann-box oracle (oracle.neumann; Sec. "Alternate boundary conditions",
Eq. bcadjust carried over to Neumann data)."""
import numpy as np
import pytest

from oracle import neumann

L = 1.0


def grad_xyz(x):
    return np.stack([x[:, 1] * x[:, 2], x[:, 0] * x[:, 2], x[:, 0] * x[:, 1]], axis=1)


def grad_cubic(x):
    return np.stack([3 * x[:, 0] ** 2 - 3 * x[:, 1] ** 2, -6 * x[:, 0] * x[:, 1], np.ones(len(x))], axis=1)


@pytest.mark.parametrize("g, grad", [(lambda x: x[:, 0] * x[:, 1] * x[:, 2], grad_xyz),
                                     (lambda x: x[:, 0] ** 3 - 3 * x[:, 0] * x[:, 1] ** 2 + x[:, 2], grad_cubic)])
def test_harmonic_flux_in_the_fe_space_is_reproduced(g, grad):
    # no charge and the normal derivative of a harmonic polynomial of the Q3 space: the
    # Galerkin solution is that polynomial up to the constant the data leaves free
    probes = np.random.default_rng(5).uniform(0, L, size=(30, 3))
    f = neumann.forward(probes, np.zeros(len(probes)), L, 6, lambda x, nr: np.einsum('mk,mk->m', grad(x), nr),
                        n_sr=2)
    d = f['phi'] - g(probes)
    assert np.abs(d - d.mean()).max() < 1e-12


@pytest.fixture(scope="module")
def free_space():
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, L, size=(80, 3))
    Q = rng.choice([-1.0, 1.0], size=80)
    D = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(D, np.inf)
    ref = (Q[None, :] / D).sum(axis=1)

    def gn(x, nr):                                            # outward flux of the free-space potential
        rel = x[:, None, :] - pos[None, :, :]
        R = np.linalg.norm(rel, axis=2)
        return (-Q[None, :] * np.einsum('mjk,mk->mj', rel, nr) / R ** 3).sum(axis=1)
    return pos, Q, gn, ref


def shifted_error(phi, ref):
    d = phi - ref
    d -= d.mean()                                             # Neumann data fixes Phi up to a constant
    return np.linalg.norm(d) / np.linalg.norm(ref)


def test_free_space_flux_gives_the_direct_sum(free_space):
    # measured 8.3e-3 (n_sr = 2) and 4.7e-3 (n_sr = 3) at n = 8
    pos, Q, gn, ref = free_space
    err = {n_sr: shifted_error(neumann.forward(pos, Q, L, 8, gn, n_sr=n_sr)['phi'], ref) for n_sr in (2, 3)}
    assert err[3] < err[2] < 1.5e-2, err


def test_boundary_adjustment_is_needed(free_space):
    pos, Q, gn, ref = free_space
    assert shifted_error(neumann.forward(pos, Q, L, 8, gn, n_sr=2, adjust=False)['phi'], ref) > 0.3
