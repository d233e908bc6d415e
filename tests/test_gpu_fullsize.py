"""Parity at the full workload sizes, in the launch configuration bench.py times
(FEP3M(L, n_el, precision) -> set_particles -> compute(forces=True)).

* jittered rock salt 32^3 / 32^3 mesh (the bench workload): against the stored
  oracle sample (tests/golden/nacl32_sample.txt, written by the oracle alone);
* 262 144 uniform charges / 64^3 mesh: the oracle's Phi at 64 sampled charges,
  central finite differences of the FP64 U for the forces, exact invariance
  under a whole-element shift of every charge;
* 999 999 water atoms / 128^3 mesh and 4 000 000 clustered charges / 256^3
  mesh: the mixed path against the FP64 path on every charge;
* oracle samples at 64 charges: Phi on all three large workloads, forces
  (the oracle's adjoint at those charges) on the uniform and water ones, and
  the Ewald force on the uniform one (the method's own error).

Tolerances: FP64 max|dPhi| / max|Phi| <= 1e-11; mixed relative RMS 1e-6 (Phi)
and 1e-5 (forces), relative error 2e-6 in U.
"""
import os

import numpy as np
import pytest

from oracle import ewald as oew
from oracle import fep3m as ofe
from paper_1503_08509_gb300 import workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
U_TOL = 2e-6   # relative error of the mixed path's U (see test_gpu_parity.py)


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


def run(api, d, precision, forces=True, pos=None):
    import torch
    eng = api.FEP3M(d["L"], d["n_el"], precision=precision)
    eng.set_particles(torch.tensor(d["pos"] if pos is None else pos, device="cuda"),
                      torch.tensor(d["Q"], device="cuda"))
    out = eng.compute(forces=forces)
    res = dict(phi=out["phi"].cpu().numpy(), U=out["U"])
    if forces:
        res["F"] = out["forces"].cpu().numpy()
    del eng
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------- rock salt 32^3
def nacl32_sample():
    path = os.path.join(HERE, "golden", "nacl32_sample.txt")
    with open(path) as fh:
        hdr = [next(fh) for _ in range(3)]
    U = float(hdr[1].split()[-1])
    a = np.loadtxt(path)
    return dict(idx=a[:, 0].astype(int), phi=a[:, 5], F=a[:, 6:9], U=U)


@pytest.fixture(scope="module")
def nacl32(api):
    d = workloads.workload("nacl32")
    return d, nacl32_sample(), run(api, d, "fp64"), run(api, d, "mixed")


def test_nacl32_fp64_matches_oracle(nacl32):
    d, ref, r64, _ = nacl32
    i = ref["idx"]
    assert maxrel(r64["phi"][i], ref["phi"]) < 1e-11, maxrel(r64["phi"][i], ref["phi"])
    assert abs(r64["U"] - ref["U"]) < 1e-11 * abs(ref["U"])
    assert maxrel(r64["F"][i], ref["F"]) < 1e-10, maxrel(r64["F"][i], ref["F"])


def test_nacl32_mixed_matches_oracle(nacl32):
    d, ref, _, r32 = nacl32
    i = ref["idx"]
    assert normrel(r32["phi"][i], ref["phi"]) < 1e-6, normrel(r32["phi"][i], ref["phi"])
    assert abs(r32["U"] - ref["U"]) < U_TOL * abs(ref["U"]), abs(r32["U"] - ref["U"]) / abs(ref["U"])


def test_nacl32_mixed_forces_match_oracle(nacl32):
    # rock-salt forces are small residues of field parts about seven times larger,
    # so this is the tightest case for the FP32 path
    _, ref, _, r32 = nacl32
    i = ref["idx"]
    assert normrel(r32["F"][i], ref["F"]) < 1e-5, normrel(r32["F"][i], ref["F"])


def test_nacl32_mixed_forces_match_fp64(nacl32):
    _, _, r64, r32 = nacl32
    assert normrel(r32["F"], r64["F"]) < 1e-5, normrel(r32["F"], r64["F"])


# --------------------------------------------------------- uniform 262k / 64^3
@pytest.fixture(scope="module")
def w4(api):
    d = workloads.workload("uniform262k")
    return d, run(api, d, "fp64"), run(api, d, "mixed")


@pytest.mark.slow
def test_uniform262k_matches_oracle_sample(w4):
    d, r64, r32 = w4
    tg = np.sort(np.random.default_rng(7).choice(len(d["Q"]), 64, replace=False))
    ref = ofe.forward(d["pos"], d["Q"], d["L"], d["n_el"], targets=tg)
    assert maxrel(r64["phi"][tg], ref["phi"]) < 1e-11, maxrel(r64["phi"][tg], ref["phi"])
    assert normrel(r32["phi"][tg], ref["phi"]) < 1e-6, normrel(r32["phi"][tg], ref["phi"])


@pytest.mark.slow
def test_uniform262k_forces_match_oracle_sample(w4):
    """Forces at 64 sampled charges against the oracle's (the energy's adjoint at
    those charges, with both mesh solves over every charge)."""
    d, r64, r32 = w4
    tg = np.sort(np.random.default_rng(9).choice(len(d["Q"]), 64, replace=False))
    F = ofe.forces_at(d["pos"], d["Q"], d["L"], d["n_el"], tg)
    assert maxrel(r64["F"][tg], F) < 1e-10, maxrel(r64["F"][tg], F)
    assert normrel(r32["F"][tg], F) < 1e-5, normrel(r32["F"][tg], F)


@pytest.mark.slow
def test_uniform262k_forces_against_ewald(w4):
    """The Ewald force at 64 sampled charges as the reference of the method itself:
    both precisions carry the same discretisation error (q = 1, 7^3 block, h = L/64;
    the oracle's is 6.0e-3 relative RMS on these charges), far above the mixed
    path's own rounding."""
    d, r64, r32 = w4
    tg = np.sort(np.random.default_rng(10).choice(len(d["Q"]), 64, replace=False))
    _, grad = oew.ewald(d["pos"], d["Q"], d["L"], targets=tg, want_grad=True)
    Fe = -d["Q"][tg, None] * grad
    e64, e32 = normrel(r64["F"][tg], Fe), normrel(r32["F"][tg], Fe)
    assert e64 < 1e-2, e64
    assert abs(e32 - e64) < 1e-3 * e64, (e32, e64)


def test_uniform262k_mixed_matches_fp64(w4):
    d, r64, r32 = w4
    assert normrel(r32["phi"], r64["phi"]) < 1e-6, normrel(r32["phi"], r64["phi"])
    assert normrel(r32["F"], r64["F"]) < 1e-5, normrel(r32["F"], r64["F"])


def test_uniform262k_forces_are_minus_grad_U(api, w4):
    """F = -dU/dx by central differences of the FP64 U (h = 1e-5 L) at 64
    charges at least 2h from every element face (U is smooth there)."""
    import torch
    d, r64, _ = w4
    L, n = d["L"], d["n_el"]
    hfd = 1e-5 * L
    t = np.mod(d["pos"] / (L / n), 1.0)
    far = np.all((t > 2 * hfd * n / L) & (t < 1 - 2 * hfd * n / L), axis=1)
    pick = np.random.default_rng(8).choice(np.flatnonzero(far), 64, replace=False)
    eng = api.FEP3M(L, n, precision="fp64")
    Qd = torch.tensor(d["Q"], device="cuda")
    base = torch.tensor(d["pos"], device="cuda")
    fd = np.zeros((len(pick), 3))
    for a, i in enumerate(pick):
        for k in range(3):
            u = []
            for s in (1.0, -1.0):
                p = base.clone()
                p[i, k] += s * hfd
                eng.set_particles(p, Qd)
                u.append(eng.compute(forces=False)["U"])
            fd[a, k] = -(u[0] - u[1]) / (2 * hfd)
    del eng
    torch.cuda.empty_cache()
    assert normrel(r64["F"][pick], fd) < 1e-5, normrel(r64["F"][pick], fd)


def test_uniform262k_whole_element_shift_invariance(api, w4):
    d, r64, _ = w4
    h = d["L"] / d["n_el"]
    shifted = d["pos"] + np.array([h, -2 * h, 3 * h])
    r = run(api, d, "fp64", pos=shifted)
    assert maxrel(r["phi"], r64["phi"]) < 1e-12, maxrel(r["phi"], r64["phi"])
    assert maxrel(r["F"], r64["F"]) < 1e-11, maxrel(r["F"], r64["F"])


# ------------------------------------------------ water 1M / 128^3, blobs 4M / 256^3
@pytest.mark.slow
@pytest.mark.parametrize("name", ["water1m", "blobs4m"])
def test_large_mixed_matches_fp64(api, name):
    d = workloads.workload(name)
    r64 = run(api, d, "fp64")
    r32 = run(api, d, "mixed")
    assert np.isfinite(r64["phi"]).all() and np.isfinite(r64["F"]).all()
    assert normrel(r32["phi"], r64["phi"]) < 1e-6, normrel(r32["phi"], r64["phi"])
    assert normrel(r32["F"], r64["F"]) < 1e-5, normrel(r32["F"], r64["F"])
    assert abs(r32["U"] - r64["U"]) < U_TOL * abs(r64["U"]), abs(r32["U"] - r64["U"]) / abs(r64["U"])


@pytest.mark.slow
def test_blobs4m_matches_oracle_sample(api):
    d = workloads.workload("blobs4m")
    tg = np.sort(np.random.default_rng(7).choice(len(d["Q"]), 64, replace=False))
    ref = ofe.forward(d["pos"], d["Q"], d["L"], d["n_el"], targets=tg)
    r64 = run(api, d, "fp64", forces=False)
    r32 = run(api, d, "mixed", forces=False)
    assert maxrel(r64["phi"][tg], ref["phi"]) < 1e-11, maxrel(r64["phi"][tg], ref["phi"])
    assert normrel(r32["phi"][tg], ref["phi"]) < 1e-6, normrel(r32["phi"][tg], ref["phi"])


@pytest.mark.slow
def test_water1m_forces_match_oracle_sample(api):
    d = workloads.workload("water1m")
    tg = np.sort(np.random.default_rng(11).choice(len(d["Q"]), 64, replace=False))
    F = ofe.forces_at(d["pos"], d["Q"], d["L"], d["n_el"], tg)
    r64 = run(api, d, "fp64")
    r32 = run(api, d, "mixed")
    assert maxrel(r64["F"][tg], F) < 1e-10, maxrel(r64["F"][tg], F)
    assert normrel(r32["F"][tg], F) < 1e-5, normrel(r32["F"][tg], F)


@pytest.mark.slow
def test_water1m_matches_oracle_sample(api):
    d = workloads.workload("water1m")
    tg = np.sort(np.random.default_rng(7).choice(len(d["Q"]), 64, replace=False))
    ref = ofe.forward(d["pos"], d["Q"], d["L"], d["n_el"], targets=tg)
    r64 = run(api, d, "fp64", forces=False)
    r32 = run(api, d, "mixed", forces=False)
    assert maxrel(r64["phi"][tg], ref["phi"]) < 1e-11, maxrel(r64["phi"][tg], ref["phi"])
    assert normrel(r32["phi"][tg], ref["phi"]) < 1e-6, normrel(r32["phi"][tg], ref["phi"])
