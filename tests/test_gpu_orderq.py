"""Screens of order q >= 2 on the order p = q + 2 mesh (Sec. 2.1, Sec. 2.4, the
Remark of Sec. 4) and one-element screens (Sec. 5.3): the CUDA path against the
order-q oracle stage by stage, and the error against Ewald on the paper's
two-cube workload falling with q (Sec. 4, Fig. compareerr).

Tolerances: FP64 max|d| / max|ref| 1e-11 (potentials, mesh solution), the
stage arrays to rounding; mixed relative RMS 1e-6 in Phi, 2e-6 relative in U.
"""
import numpy as np
import pytest

from oracle import ewald, highorder
from paper_1503_08509_gb300 import workloads

pytestmark = pytest.mark.gpu

PAD = 2           # the library's default table margin for q >= 2 (half width n_sr + 1 + PAD)
NGL = 8           # Gauss-Legendre points per piece of the tables' boundary quadrature, as the library


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


CASE = dict(zip(("pos", "Q"), workloads.uniform_pm(300, seed=13)), L=1.3, n_el=8)
_ref = {}


def oracle(q, support):
    if (q, support) not in _ref:
        d = CASE
        _ref[(q, support)] = highorder.forward(d["pos"], d["Q"], d["L"], d["n_el"], q, n_sr=3,
                                               half_width=3 + 1 + PAD, ngl=NGL, support=support)
    return _ref[(q, support)]


def run(api, q, support, precision):
    import torch
    d = CASE
    eng = api.FEP3M(d["L"], d["n_el"], precision=precision, q=q, one_element=support == "element")
    eng.set_particles(torch.tensor(d["pos"], device="cuda"), torch.tensor(d["Q"], device="cuda"))
    out = eng.compute(forces=False)
    return eng, out


@pytest.mark.parametrize("q,support", [(2, "patch"), (3, "patch"), (2, "element"), (3, "element")])
def test_fp64_stages_match_oracle(api, q, support):
    ref = oracle(q, support)
    eng, out = run(api, q, support, "fp64")
    h = CASE["L"] / CASE["n_el"]
    m = eng.mesh()
    C = ref["C"] * h ** 3
    assert np.abs(m["C"] - C).max() < 1e-13 * np.abs(C).max()
    b = ref["b"].transpose(2, 1, 0).ravel()
    assert np.abs(m["b"] - b).max() < 1e-12 * np.abs(b).max()
    pm = ref["phi_mesh"].transpose(2, 1, 0).ravel()
    assert maxrel(m["phi_mesh"], pm) < 1e-11, maxrel(m["phi_mesh"], pm)
    phi = out["phi"].cpu().numpy()
    assert maxrel(phi, ref["phi"]) < 1e-11, maxrel(phi, ref["phi"])
    assert abs(out["U"] - ref["U"]) < 1e-11 * abs(ref["U"])
    st = eng.stats()
    assert st["mg_rel_residual"] <= 1e-12, st


@pytest.mark.parametrize("q,support", [(2, "patch"), (3, "patch"), (2, "element")])
def test_mixed_matches_oracle(api, q, support):
    ref = oracle(q, support)
    _, out = run(api, q, support, "mixed")
    phi = out["phi"].cpu().numpy()
    assert normrel(phi, ref["phi"]) < 1e-6, normrel(phi, ref["phi"])
    assert abs(out["U"] - ref["U"]) < 2e-6 * abs(ref["U"]), abs(out["U"] - ref["U"]) / abs(ref["U"])


@pytest.mark.parametrize("q", [2, 3])
def test_order_p_mesh_solve(api, q):
    """The order-p solve alone (refinement around the FP32 fast-diagonalisation
    solve) against the oracle's exact solve, on a random neutral right-hand side
    over a mesh whose node count is not a multiple of the transform tiles."""
    n = 9
    ops = highorder.MeshOperators(1.7, n, q + 2, q)
    rng = np.random.default_rng(q)
    b = ops.neutralise(rng.normal(size=((q + 2) * n,) * 3))
    ref = ops.solve(b)
    for precision, tol in (("fp64", 1e-11), ("mixed", 1e-7)):
        eng = api.FEP3M(1.7, n, precision=precision, q=q)
        phi = eng.solve_mesh(b.transpose(2, 1, 0).ravel())
        assert maxrel(phi, ref.transpose(2, 1, 0).ravel()) < tol, (precision, eng.stats())


def test_forces_need_order_one(api):
    import torch
    from paper_1503_08509_gb300 import _lib
    eng, _ = run(api, 2, "patch", "fp64")
    with pytest.raises(_lib.FEP3MError) as e:
        eng.compute(forces=True)
    assert e.value.status == _lib.FEP3M_EINVAL
    with pytest.raises(_lib.FEP3MError) as e:
        eng.vjp(1.0)
    assert e.value.status == _lib.FEP3M_EINVAL


@pytest.mark.slow
def test_error_falls_with_q_on_the_paper_workload(api):
    """Sec. 4, Fig. compareerr: two biased cubes, h = 1/15, 7^3 block.  The error
    against a converged Ewald sum falls with each step of q, and faster at each
    step (the oracle measured 2.9e-3, 3.2e-4, 2.3e-5, 1.5e-6 for q = 1 .. 4 on
    120 charges)."""
    import torch
    pos, Q = workloads.two_biased_cubes(1000)
    pe = ewald.ewald(pos, Q, 1.0)
    err = []
    for q in (1, 2, 3, 4):
        eng = api.FEP3M(1.0, 15, precision="fp64", q=q)
        eng.set_particles(torch.tensor(pos, device="cuda"), torch.tensor(Q, device="cuda"))
        d = eng.compute(forces=False)["phi"].cpu().numpy() - pe
        d -= d.mean()
        err.append(np.linalg.norm(d) / np.linalg.norm(pe))
        eng.close()
    gain = [err[i] / err[i + 1] for i in range(3)]
    assert err[0] < 5e-3 and gain[0] > 5 and gain[1] > gain[0] and gain[2] > gain[1], (err, gain)
