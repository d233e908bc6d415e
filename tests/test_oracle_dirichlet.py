"""Pins for the Dirichlet-box oracle (oracle.dirichlet; Sec. "Alternate boundary
conditions", Eq. bcadjust)."""
import numpy as np
import pytest

from oracle import dirichlet, fep3m

L = 1.0


@pytest.mark.parametrize("g", [lambda x: x[:, 0] * x[:, 1] * x[:, 2],
                               lambda x: x[:, 0] ** 2 - x[:, 1] ** 2 + 0.3,
                               lambda x: x[:, 0] ** 3 - 3 * x[:, 0] * x[:, 1] ** 2 + x[:, 2]])
def test_harmonic_data_in_the_fe_space_is_reproduced(g):
    # with no charge the potential is the harmonic function with boundary values g;
    # for a harmonic polynomial of degree <= 3 per variable the order-3 Galerkin
    # solution is that polynomial, at every point of the box
    probes = np.random.default_rng(5).uniform(0, L, size=(30, 3))
    f = dirichlet.forward(probes, np.zeros(len(probes)), L, 8, g, n_sr=2)
    assert np.abs(f['phi'] - g(probes)).max() < 1e-12
    pts = np.random.default_rng(6).uniform(0, L, size=(20, 3))
    assert np.abs(dirichlet.evaluate_mesh(f['phi_mesh'], pts, L, 8) - g(pts)).max() < 1e-12


@pytest.fixture(scope="module")
def free_space():
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, L, size=(80, 3))
    Q = rng.choice([-1.0, 1.0], size=80)
    D = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(D, np.inf)
    ref = (Q[None, :] / D).sum(axis=1)                       # direct free-space pair sum

    def g(x):
        return (Q[None, :] / np.linalg.norm(x[:, None, :] - pos[None, :, :], axis=2)).sum(axis=1)
    return pos, Q, g, ref


def test_free_space_data_gives_the_direct_sum(free_space):
    # Dirichlet data = the free-space potential of the charges: Phi at each charge is
    # the direct sum over the others, up to the method's truncation and FE error,
    # which falls as the short-range block grows
    pos, Q, g, ref = free_space
    err = {}
    for n_sr in (2, 3):
        f = dirichlet.forward(pos, Q, L, 8, g, n_sr=n_sr)
        err[n_sr] = np.linalg.norm(f['phi'] - ref) / np.linalg.norm(ref)
    assert err[3] < err[2] < 5e-3, err


def test_boundary_adjustment_is_needed(free_space):
    # without Eq. bcadjust the short-range potential of charges near the faces is
    # counted twice on the boundary
    pos, Q, g, ref = free_space
    f = dirichlet.forward(pos, Q, L, 8, g, n_sr=2, adjust=False)
    assert np.linalg.norm(f['phi'] - ref) / np.linalg.norm(ref) > 0.1


def interior_set(n, n_sr, N, seed):
    # charges at least n_sr + 1 elements from every face: no block reaches the boundary
    rng = np.random.default_rng(seed)
    lo, hi = (n_sr + 1) / n, 1 - (n_sr + 1) / n
    return rng.uniform(lo, hi, size=(N, 3)) * L, rng.choice([-1.0, 1.0], size=N)


def test_no_adjustment_for_charges_away_from_the_boundary():
    n, n_sr = 12, 2
    pos, Q = interior_set(n, n_sr, 40, 7)
    g = lambda x: 0.1 * x[:, 0]
    a = dirichlet.forward(pos, Q, L, n, g, n_sr=n_sr)
    b = dirichlet.forward(pos, Q, L, n, g, n_sr=n_sr, adjust=False)
    assert np.array_equal(a['phi_mesh'], b['phi_mesh'])


def test_short_range_part_matches_the_periodic_oracle():
    # away from the faces the cut-off block and the periodic block hold the same
    # charges, so the short-range parts agree (singular sum minus screens, own screen
    # included)
    n, n_sr = 12, 2
    pos, Q = interior_set(n, n_sr, 40, 8)
    f = dirichlet.forward(pos, Q, L, n, lambda x: np.zeros(len(x)), n_sr=n_sr)
    p = fep3m.forward(pos, Q, L, n, n_sr=n_sr)
    ref = p['phi_sing'] - p['phi_scr']
    assert np.abs(f['phi_sr'] - ref).max() < 1e-12 * np.abs(ref).max()
