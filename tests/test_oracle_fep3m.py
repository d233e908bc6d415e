"""Pins for the whole method as the oracle computes it (Algorithm 1, Sec. 2.1-2.5, Sec. 4)."""
import itertools

import numpy as np
import pytest

from oracle import ewald, fep3m, tables
from paper_1503_08509_gb300 import workloads


def small_set(N=240, seed=21):
    return workloads.uniform_pm(N, seed=seed)


def test_binning_rules():
    L, n = 2.0, 8
    h = L / n
    pos = np.array([[0.0, 1.999999999, -0.1], [2.0, 0.25, 4.3], [0.25 - 1e-17, 0.5, 1.0]])
    b = fep3m.bin_particles(pos, L, n)
    assert np.all(b['delta'] >= -h / 2) and np.all(b['delta'] < h / 2)
    assert tuple(b['c3'][0]) == (0, 7, 7)        # -0.1 wraps to 1.9
    assert tuple(b['c3'][1]) == (0, 1, 1)        # x = L wraps to 0; 0.25 starts element 1
    pos, Q = small_set(500)
    b = fep3m.bin_particles(pos, 1.0, 7)
    srt = b['cell'][b['perm']]
    assert np.all(np.diff(srt) >= 0)
    same = np.diff(srt) == 0
    assert np.all(np.diff(b['perm'])[same] > 0)  # stable: original order within an element


def test_shift_by_whole_elements_is_exact():
    pos, Q = small_set()
    L, n = 1.0, 8
    a = fep3m.forward(pos, Q, L, n)
    b = fep3m.forward(pos + np.array([3, -2, 5]) * (L / n), Q, L, n)
    assert np.abs(a['phi'] - b['phi']).max() < 1e-11 * np.abs(a['phi']).max()


def test_reflection_and_axis_permutation():
    pos, Q = small_set()
    L, n = 1.0, 8
    a = fep3m.forward(pos, Q, L, n)
    r = fep3m.forward(np.mod(-pos, L), Q, L, n)
    assert np.abs(a['phi'] - r['phi']).max() < 1e-11 * np.abs(a['phi']).max()
    pm = fep3m.forward(pos[:, [2, 0, 1]], Q, L, n)
    assert np.abs(a['phi'] - pm['phi']).max() < 1e-11 * np.abs(a['phi']).max()


def test_linear_in_charge():
    pos, Q = small_set()
    a = fep3m.forward(pos, Q, 1.0, 8)
    b = fep3m.forward(pos, 2 * Q, 1.0, 8)
    assert np.allclose(b['phi'], 2 * a['phi'], rtol=1e-13, atol=1e-12)
    assert abs(b['U'] - 4 * a['U']) < 1e-12 * abs(b['U'])


def test_singular_part_brute_force():
    # all pairs whose elements differ by at most n_sr per axis (periodically), j != i
    pos, Q = small_set(120, seed=5)
    L, n, n_sr = 1.0, 9, 3
    f = fep3m.forward(pos, Q, L, n)
    c3 = np.floor(np.mod(pos, L) * n / L).astype(int)
    ref = np.zeros(len(Q))
    for i, j in itertools.product(range(len(Q)), repeat=2):
        if i == j:
            continue
        d = (c3[j] - c3[i] + n // 2) % n - n // 2
        if np.all(np.abs(d) <= n_sr):
            rel = pos[j] - pos[i]
            rel -= L * np.round(rel / L)
            ref[i] += Q[j] / np.linalg.norm(rel)
    assert np.abs(f['phi_sing'] - ref).max() < 1e-12 * np.abs(ref).max()


def test_screen_part_close_to_continuum_screens():
    # each charge of the block subtracts its screen potential; with the continuum potential of
    # the screen (Eq. screenintegral) instead of the FE table the result moves only by FE error
    pos, Q = small_set(60, seed=6)
    L, n, n_sr = 1.0, 8, 3
    h = L / n
    f = fep3m.forward(pos, Q, L, n)
    b = f['bins']
    from oracle import screens
    c = screens.screen_coefficients(1, h, b['delta']) * h ** 3
    ref = np.zeros(len(Q))
    for i in range(len(Q)):
        for j in range(len(Q)):
            d = (b['c3'][j] - b['c3'][i] + n // 2) % n - n // 2
            if not np.all(np.abs(d) <= n_sr):
                continue
            for kap in range(8):
                v = d + fep3m.corner(kap) - 0.5          # vertex relative to the target element centre
                x = (b['delta'][i] - v * h) / h
                ref[i] += Q[j] * c[j, kap] * h ** 2 * tables.hat_potential_continuum(x[None, :])[0] / h ** 3
    # tensor Gauss-Legendre is inaccurate for targets inside a hat's support (singular
    # integrand), so this only pins the structure: a wrong offset, sign or corner gives O(1)
    err = np.abs(f['phi_scr'] - ref).max() / np.abs(ref).max()
    assert err < 2e-2, err


def test_rock_salt_madelung_closed_form():
    # ions on the element vertices: the method reproduces the Madelung potential M/a
    from test_oracle_ewald import madelung_nacl_benson
    m = 16
    pos, Q = workloads.rock_salt(m, jitter=0.0)
    f = fep3m.forward(pos, Q, 1.0, m)
    ref = -madelung_nacl_benson() * m * Q
    assert np.abs(f['phi'] - ref).max() < 2e-6 * np.abs(ref).max()


@pytest.fixture(scope="module")
def uniform_vs_ewald():
    pos, Q = workloads.uniform_pm(400, seed=9)
    pe, ge = ewald.ewald(pos, Q, 1.0, want_grad=True)
    return pos, Q, pe, ge


def normwise_shifted(phi, ref):
    d = phi - ref
    d -= d.mean()            # the potentials may differ by a constant (Sec. 4)
    return np.linalg.norm(d) / np.linalg.norm(ref)


def test_accuracy_against_ewald(uniform_vs_ewald):
    pos, Q, pe, _ = uniform_vs_ewald
    errs = {}
    for n_sr in (2, 4):
        f = fep3m.forward(pos, Q, 1.0, 12, n_sr=n_sr)
        errs[n_sr] = normwise_shifted(f['phi'], pe)
        assert abs(f['U'] - 0.5 * Q @ pe) < 2e-2 * abs(0.5 * Q @ pe)
    assert errs[4] < errs[2] < 2e-2, errs


def test_forces_against_ewald(uniform_vs_ewald):
    pos, Q, _, ge = uniform_vs_ewald
    f = fep3m.forward(pos, Q, 1.0, 12, want_grad=True)
    dx, _, _ = fep3m.vjp(f, Q)
    ref = Q[:, None] * ge                           # dU/dx from Ewald
    assert np.linalg.norm(dx - ref) / np.linalg.norm(ref) < 5e-2


def test_momentum_is_not_conserved_exactly(uniform_vs_ewald):
    # Sec. 5.3: the method's operators lack the symmetry that makes pair forces cancel,
    # so the forces -dU/dx do not sum to zero exactly (they do for Ewald, to rounding);
    # measured sum |F| ratio 4.0e-4 here.  The field forces Q E(x) (no source-side
    # derivative of the screens) are closer to Ewald: 4.2e-3 against 1.6e-2.
    pos, Q, _, ge = uniform_vs_ewald
    f = fep3m.forward(pos, Q, 1.0, 12, n_sr=2, want_grad=True)
    dx, _, _ = fep3m.vjp(f, Q, n_sr=2)
    ref = Q[:, None] * ge
    drift = np.linalg.norm(dx.sum(axis=0)) / np.abs(dx).sum()
    assert 1e-6 < drift < 1e-2, drift
    assert np.linalg.norm(ref.sum(axis=0)) < 1e-12 * np.abs(ref).sum()
    field = Q[:, None] * f['grad_field']
    assert np.linalg.norm(field - ref) < np.linalg.norm(dx - ref)


def face_safe(pos, L, n, margin):
    t = np.mod(pos, L) * n / L
    frac = t - np.floor(t)
    return np.all((frac > margin * n / L) & (frac < 1 - margin * n / L), axis=1)


def test_adjoint_against_central_differences():
    pos, Q = small_set(150, seed=31)
    L, n = 1.0, 8
    f = fep3m.forward(pos, Q, L, n, want_grad=True)
    rng = np.random.default_rng(2)
    gphi = rng.normal(size=len(Q))
    dx, dQ, _ = fep3m.vjp(f, Q, gU=0.7, gphi=gphi)

    def loss(p, q):
        g = fep3m.forward(p, q, L, n)
        return 0.7 * g['U'] + gphi @ g['phi']
    hfd = 1e-5 * L
    cand = np.where(face_safe(pos, L, n, 4 * hfd))[0][:4]
    for i in cand:
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += hfd
            pm[i, a] -= hfd
            fd = (loss(pp, Q) - loss(pm, Q)) / (2 * hfd)
            assert abs(fd - dx[i, a]) < 1e-6 * max(1.0, abs(fd)), (i, a, fd, dx[i, a])
        qp, qm = Q.copy(), Q.copy()
        qp[i] += 1e-5
        qm[i] -= 1e-5
        fd = (loss(pos, qp) - loss(pos, qm)) / 2e-5
        assert abs(fd - dQ[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, dQ[i])


def test_forces_at_sampled_charges():
    """forces_at (the energy's adjoint restricted to some charges, with the mesh
    solves over every charge) equals -dU/dx by central differences of U at those
    charges, and the full adjoint there."""
    pos, Q = small_set(180, seed=41)
    L, n = 1.3, 9
    tg = np.sort(np.random.default_rng(5).choice(len(Q), 12, replace=False))
    F = fep3m.forces_at(pos, Q, L, n, tg)
    f = fep3m.forward(pos, Q, L, n, want_grad=True)
    dx, _, _ = fep3m.vjp(f, Q)
    assert np.abs(F + dx[tg]).max() < 1e-12 * np.abs(dx).max()
    hfd = 1e-5 * L
    safe = [k for k, i in enumerate(tg) if face_safe(pos[i:i + 1], L, n, 4 * hfd)[0]][:3]
    for k in safe:
        i = tg[k]
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += hfd
            pm[i, a] -= hfd
            fd = -(fepu(pp, Q, L, n) - fepu(pm, Q, L, n)) / (2 * hfd)
            assert abs(fd - F[k, a]) < 1e-6 * max(1.0, abs(fd)), (i, a, fd, F[k, a])


def fepu(pos, Q, L, n):
    return fep3m.forward(pos, Q, L, n)['U']
