"""Pins for the independent Ewald oracle."""
import numpy as np
import pytest

from oracle import ewald
from paper_1503_08509_gb300 import workloads


def madelung_nacl_benson(terms=40):
    """Rock-salt Madelung constant from Benson's rapidly convergent series:
    M = 12 pi sum_{m, n odd > 0} sech^2(pi/2 sqrt(m^2 + n^2))."""
    odd = np.arange(1, 2 * terms, 2)
    M, N = np.meshgrid(odd, odd)
    return 12 * np.pi * np.sum(1.0 / np.cosh(0.5 * np.pi * np.sqrt(M ** 2 + N ** 2)) ** 2)


def test_benson_series_value():
    assert abs(madelung_nacl_benson() - 1.747564594633) < 1e-12


@pytest.mark.parametrize("m", [4, 8])
def test_rock_salt_madelung(m):
    pos, Q = workloads.rock_salt(m, jitter=0.0)
    phi = ewald.ewald(pos, Q, 1.0)
    a = 1.0 / m
    assert np.abs(phi * Q * a + madelung_nacl_benson()).max() < 1e-12


def test_alpha_independence_and_forces():
    pos, Q = workloads.uniform_pm(40, seed=11)
    p1, g1 = ewald.ewald(pos, Q, 1.0, want_grad=True)
    p2, g2 = ewald.ewald(pos, Q, 1.0, alpha_L=9.0, want_grad=True)
    assert np.abs(p1 - p2).max() < 1e-12 * np.abs(p1).max()
    assert np.abs(g1 - g2).max() < 1e-11 * np.abs(g1).max()
    i, hfd = 7, 1e-6
    for a in range(3):
        pp, pm = pos.copy(), pos.copy()
        pp[i, a] += hfd
        pm[i, a] -= hfd
        fd = (ewald.ewald_energy(pp, Q, 1.0) - ewald.ewald_energy(pm, Q, 1.0)) / (2 * hfd)
        assert abs(fd - Q[i] * g1[i, a]) < 1e-6 * max(1.0, abs(fd))


def test_two_charge_near_field():
    # a close +/- pair in a big cell: Phi -> -/+1/d plus the small periodic correction
    L, d = 1.0, 1e-3
    pos = np.array([[0.5, 0.5, 0.5], [0.5 + d, 0.5, 0.5]])
    Q = np.array([1.0, -1.0])
    phi = ewald.ewald(pos, Q, L)
    assert abs(phi[0] + 1.0 / d) < 1e-2 and abs(phi[1] - 1.0 / d) < 1e-2
    assert abs(phi[0] + phi[1]) < 1e-12
