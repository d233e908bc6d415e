"""The box [0, L]^3 with Dirichlet or Neumann data (Sec. "Alternate boundary
conditions", Eq. bcadjust): the CUDA path against the Dirichlet and Neumann
oracles stage by stage, the mesh solves alone against the oracles' exact
solves, and two properties the paper's construction fixes without any oracle:
harmonic data of degree <= 3 per variable is reproduced exactly (Neumann: up to
a constant), and free-space data gives the direct pair sum up to the method's
error.

Tolerances: FP64 max|d| / max|ref| 1e-11 (potentials, mesh solution) and the
stage arrays to rounding; mixed relative RMS 1e-6 in Phi, 2e-6 relative in U
(those of the periodic path).
"""
import numpy as np
import pytest

from oracle import dirichlet
from paper_1503_08509_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08509_gb300 import api as a, build
    build.build()
    return a


def maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def normrel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def g_smooth(x):
    """Dirichlet data that is not harmonic and not in the FE space."""
    return 0.4 + 0.3 * x[:, 0] - 0.2 * x[:, 1] ** 2 + 0.1 * np.sin(2.0 * x[:, 2]) + 0.05 * x[:, 0] * x[:, 1]


L, NEL, NSR = 1.3, 8, 3
POS, Q = workloads.box_charges(300, L=L, seed=7)
_ref = {}


def oracle():
    if "f" not in _ref:
        _ref["f"] = dirichlet.forward(POS, Q, L, NEL, g_smooth, n_sr=NSR)
    return _ref["f"]


def run(api, precision, tensor_cores=True, pos=POS, Qv=Q, g=g_smooth, n_el=NEL, n_sr=NSR, Lb=L):
    import torch
    eng = api.FEP3M(Lb, n_el, n_sr=n_sr, precision=precision, dirichlet=True, tensor_cores=tensor_cores)
    eng.set_boundary(g(eng.node_points()))
    eng.set_particles(torch.tensor(pos, device="cuda"), torch.tensor(Qv, device="cuda"))
    return eng, eng.compute(forces=False)


def test_binning_bit_exact(api):
    import torch
    ref = dirichlet.bin_box(POS, L, NEL)
    eng = api.FEP3M(L, NEL, n_sr=NSR, precision="fp64", dirichlet=True)
    eng.set_particles(torch.tensor(POS, device="cuda"), torch.tensor(Q, device="cuda"))
    b = eng.binning()
    c3 = ref["c3"]
    cell = c3[:, 0] + NEL * (c3[:, 1] + NEL * c3[:, 2])
    assert np.array_equal(b["cell"], cell)
    assert np.array_equal(b["count"], np.bincount(cell, minlength=NEL ** 3))
    assert np.array_equal(b["perm"], np.argsort(cell, kind="stable"))
    assert np.array_equal(b["delta"], ref["delta"])
    # the faces x = L belong to the last element, at offset +h/2
    onL = np.flatnonzero(POS == L)
    assert len(onL) > 0 and np.all(c3[POS == L] == NEL - 1)


def test_fp64_stages_match_oracle(api):
    ref = oracle()
    eng, out = run(api, "fp64")
    h = L / NEL
    m = eng.mesh()
    C = (ref["C"] * h ** 3).transpose(2, 1, 0, 3).reshape(-1, 8)
    assert np.abs(m["C"] - C).max() < 1e-13 * np.abs(C).max()
    b = ref["b"].transpose(2, 1, 0).ravel()
    assert np.abs(m["b"] - b).max() < 1e-12 * np.abs(b).max()
    pm = ref["phi_mesh"].transpose(2, 1, 0).ravel()
    assert maxrel(m["phi_mesh"], pm) < 1e-11, maxrel(m["phi_mesh"], pm)
    phi = out["phi"].cpu().numpy()
    assert maxrel(phi, ref["phi"]) < 1e-11, maxrel(phi, ref["phi"])
    assert abs(out["U"] - ref["U"]) < 1e-11 * abs(ref["U"])
    st = eng.stats()
    assert st["mg_rel_residual"] <= 1e-13 and st["refine_steps"] <= 4, st


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_mixed_matches_oracle(api, tensor_cores):
    ref = oracle()
    eng, out = run(api, "mixed", tensor_cores=tensor_cores)
    phi = out["phi"].cpu().numpy()
    assert normrel(phi, ref["phi"]) < 1e-6, normrel(phi, ref["phi"])
    assert abs(out["U"] - ref["U"]) < 2e-6 * abs(ref["U"]), abs(out["U"] - ref["U"]) / abs(ref["U"])
    pm = ref["phi_mesh"].transpose(2, 1, 0).ravel()
    assert maxrel(eng.mesh()["phi_mesh"], pm) < 1e-6


@pytest.mark.parametrize("n_el", [7, 9])
def test_dirichlet_mesh_solve(api, n_el):
    """The interior solve alone: random load, random boundary data, against the
    oracle's exact fast-diagonalisation solve (interior node counts 20 and 26,
    not multiples of the transform tiles)."""
    Lb = 0.9
    h = Lb / n_el
    M1, K1, _ = dirichlet.open_matrices(n_el, h)
    Nn = 3 * n_el + 1
    rng = np.random.default_rng(n_el)
    b = rng.normal(size=(Nn,) * 3)
    gnode = rng.normal(size=(Nn,) * 3)
    onb = np.zeros((Nn,) * 3, dtype=bool)
    onb[[0, -1], :, :] = onb[:, [0, -1], :] = onb[:, :, [0, -1]] = True
    phiB = np.where(onb, gnode, 0.0)
    ref = dirichlet.solve_interior(b, phiB, M1, K1)
    for precision, tol in (("fp64", 1e-11), ("mixed", 1e-8)):
        eng = api.FEP3M(Lb, n_el, n_sr=3, precision=precision, dirichlet=True)
        eng.set_boundary(gnode.transpose(2, 1, 0).ravel())
        phi = eng.solve_mesh(b.transpose(2, 1, 0).ravel())
        assert maxrel(phi, ref.transpose(2, 1, 0).ravel()) < tol, (precision, eng.stats())


def test_harmonic_data_is_reproduced(api):
    """No charge (zero charges at probe points): the potential is the harmonic
    extension of g, which the order-3 space holds exactly for a harmonic
    polynomial of degree <= 3 per variable."""
    probes = np.random.default_rng(5).uniform(0, L, size=(40, 3))

    def g(x):
        return x[:, 0] ** 3 - 3 * x[:, 0] * x[:, 1] ** 2 + x[:, 2] + x[:, 0] * x[:, 1] * x[:, 2]
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
        _, out = run(api, precision, pos=probes, Qv=np.zeros(len(probes)), g=g)
        phi = out["phi"].cpu().numpy()
        assert np.abs(phi - g(probes)).max() < tol * np.abs(g(probes)).max(), precision


def test_free_space_data_gives_the_direct_sum(api):
    """Dirichlet data = the free-space potential of the charges themselves: Phi_i
    is the direct sum over the other charges, up to the method's truncation and
    FE error (as for the oracle: below 5e-3 with n_sr = 3 on 8^3 elements)."""
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 1.0, size=(80, 3))
    Qv = rng.choice([-1.0, 1.0], size=80)
    D = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(D, np.inf)
    direct = (Qv[None, :] / D).sum(axis=1)

    def g(x):
        return (Qv[None, :] / np.linalg.norm(x[:, None, :] - pos[None, :, :], axis=2)).sum(axis=1)
    for precision in ("fp64", "mixed"):
        _, out = run(api, precision, pos=pos, Qv=Qv, g=g, n_el=8, n_sr=3, Lb=1.0)
        phi = out["phi"].cpu().numpy()
        assert normrel(phi, direct) < 5e-3, (precision, normrel(phi, direct))


def test_box_errors(api):
    import torch
    from paper_1503_08509_gb300 import _lib
    eng = api.FEP3M(L, NEL, n_sr=NSR, precision="fp64", dirichlet=True)
    bad = POS.copy()
    bad[3, 1] = L * (1 + 1e-12)
    with pytest.raises(_lib.FEP3MError) as e:
        eng.set_particles(torch.tensor(bad, device="cuda"), torch.tensor(Q, device="cuda"))
    assert e.value.status == _lib.FEP3M_EINVAL
    bad[3, 1] = -1e-300
    with pytest.raises(_lib.FEP3MError) as e:
        eng.set_particles(torch.tensor(bad, device="cuda"), torch.tensor(Q, device="cuda"))
    assert e.value.status == _lib.FEP3M_EINVAL
    g = g_smooth(eng.node_points())
    g[5] = np.nan
    with pytest.raises(_lib.FEP3MError) as e:
        eng.set_boundary(g)
    assert e.value.status == _lib.FEP3M_EINVAL
    eng.set_particles(torch.tensor(POS, device="cuda"), torch.tensor(Q, device="cuda"))
    with pytest.raises(_lib.FEP3MError) as e:
        eng.compute(forces=True)
    assert e.value.status == _lib.FEP3M_EINVAL
    with pytest.raises(_lib.FEP3MError) as e:
        eng.vjp(1.0)
    assert e.value.status == _lib.FEP3M_EINVAL
    # the box ignores neutrality: a single charge is a valid input
    eng.set_particles(torch.tensor(POS[:1], device="cuda"), torch.tensor([2.5], device="cuda"))
    out = eng.compute(forces=False)
    assert np.isfinite(out["U"])


# ------------------------------------------------------------------ Neumann data
from oracle import neumann  # noqa: E402


def gn_smooth(x, nr):
    """Outward flux data that is not the flux of a harmonic function."""
    grad = np.stack([0.3 + 0.05 * x[:, 1], -0.4 * x[:, 1] + 0.05 * x[:, 0], 0.2 * np.cos(2.0 * x[:, 2])], axis=1)
    return np.einsum('mk,mk->m', grad, nr) + 0.1 * np.sin(3.0 * x[:, 0] * x[:, 1])


def oracle_neumann():
    if "n" not in _ref:
        f = neumann.forward(POS, Q, L, NEL, gn_smooth, n_sr=NSR)
        f["U"] = 0.5 * np.dot(Q, f["phi"])
        _ref["n"] = f
    return _ref["n"]


def run_neumann(api, precision, tensor_cores=True, pos=POS, Qv=Q, gn=gn_smooth, n_el=NEL, n_sr=NSR, Lb=L):
    import torch
    eng = api.FEP3M(Lb, n_el, n_sr=n_sr, precision=precision, neumann=True, tensor_cores=tensor_cores)
    eng.set_boundary(gn(*eng.face_points()))
    eng.set_particles(torch.tensor(pos, device="cuda"), torch.tensor(Qv, device="cuda"))
    return eng, eng.compute(forces=False)


def test_neumann_fp64_stages_match_oracle(api):
    """Both sides fix the constant by int phi^sm = 0, so Phi compares directly."""
    ref = oracle_neumann()
    eng, out = run_neumann(api, "fp64")
    m = eng.mesh()
    b = ref["b"].transpose(2, 1, 0).ravel()
    assert np.abs(m["b"] - b).max() < 1e-12 * np.abs(b).max()
    pm = ref["phi_mesh"].transpose(2, 1, 0).ravel()
    assert maxrel(m["phi_mesh"], pm) < 1e-11, maxrel(m["phi_mesh"], pm)
    phi = out["phi"].cpu().numpy()
    assert maxrel(phi, ref["phi"]) < 1e-11, maxrel(phi, ref["phi"])
    assert abs(out["U"] - ref["U"]) < 1e-11 * abs(ref["U"])
    st = eng.stats()
    assert st["mg_rel_residual"] <= 1e-13 and st["refine_steps"] <= 4, st


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_neumann_mixed_matches_oracle(api, tensor_cores):
    ref = oracle_neumann()
    _, out = run_neumann(api, "mixed", tensor_cores=tensor_cores)
    phi = out["phi"].cpu().numpy()
    assert normrel(phi, ref["phi"]) < 1e-6, normrel(phi, ref["phi"])
    assert abs(out["U"] - ref["U"]) < 2e-6 * abs(ref["U"]), abs(out["U"] - ref["U"]) / abs(ref["U"])


@pytest.mark.parametrize("n_el", [7, 9])
def test_neumann_mesh_solve(api, n_el):
    """The fully Neumann solve alone (node counts 22 and 28 per axis) against the
    oracle's exact solve of the compatible load."""
    Lb = 0.9
    M1, K1, _ = dirichlet.open_matrices(n_el, Lb / n_el)
    Nn = 3 * n_el + 1
    b = np.random.default_rng(n_el + 100).normal(size=(Nn,) * 3)
    ref = neumann.solve_compatible(b, M1, K1)
    for precision, tol in (("fp64", 1e-11), ("mixed", 1e-8)):
        eng = api.FEP3M(Lb, n_el, n_sr=3, precision=precision, neumann=True)
        phi = eng.solve_mesh(b.transpose(2, 1, 0).ravel())
        assert maxrel(phi, ref.transpose(2, 1, 0).ravel()) < tol, (precision, eng.stats())


def test_neumann_harmonic_flux_is_reproduced(api):
    """No charge: the flux of a harmonic polynomial of the Q3 space gives that
    polynomial up to a constant."""
    probes = np.random.default_rng(5).uniform(0, L, size=(40, 3))

    def grad(x):
        return np.stack([3 * x[:, 0] ** 2 - 3 * x[:, 1] ** 2 + x[:, 1] * x[:, 2], -6 * x[:, 0] * x[:, 1] + x[:, 0] * x[:, 2],
                         1.0 + x[:, 0] * x[:, 1]], axis=1)

    def u(x):
        return x[:, 0] ** 3 - 3 * x[:, 0] * x[:, 1] ** 2 + x[:, 2] + x[:, 0] * x[:, 1] * x[:, 2]
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-6)):
        _, out = run_neumann(api, precision, pos=probes, Qv=np.zeros(len(probes)),
                             gn=lambda x, nr: np.einsum('mk,mk->m', grad(x), nr))
        d = out["phi"].cpu().numpy() - u(probes)
        assert np.abs(d - d.mean()).max() < tol * np.abs(u(probes)).max(), precision


def test_neumann_free_space_flux_gives_the_direct_sum(api):
    """Flux data of the charges' own free-space potential: Phi_i is the direct sum
    up to a constant and the method's error (the oracle: 4.7e-3 at n_sr = 3)."""
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 1.0, size=(80, 3))
    Qv = rng.choice([-1.0, 1.0], size=80)
    D = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(D, np.inf)
    direct = (Qv[None, :] / D).sum(axis=1)

    def gn(x, nr):
        rel = x[:, None, :] - pos[None, :, :]
        R = np.linalg.norm(rel, axis=2)
        return (-Qv[None, :] * np.einsum('mjk,mk->mj', rel, nr) / R ** 3).sum(axis=1)
    for precision in ("fp64", "mixed"):
        _, out = run_neumann(api, precision, pos=pos, Qv=Qv, gn=gn, n_el=8, n_sr=3, Lb=1.0)
        d = out["phi"].cpu().numpy() - direct
        d -= d.mean()
        assert np.linalg.norm(d) / np.linalg.norm(direct) < 1e-2, precision
