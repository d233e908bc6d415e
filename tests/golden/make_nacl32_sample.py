"""Write nacl32_sample.txt: oracle FE-P3M and Ewald values for a seeded sample of the
jittered rock-salt workload (32^3 ions, jitter 1e-3 L, 32^3 mesh).

Calls only oracle/ (and the seeded workload generator).  The Ewald sum is the
paper's comparison reference (Sec. 4), converged far below its printed settings.
Columns: index, Phi_ewald, F_ewald (3), Phi_fep3m, F_fep3m (3).  Header lines
hold U of the FE-P3M oracle and of the closed-form Madelung lattice.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ewald, fep3m  # noqa: E402
from paper_1503_08509_gb300 import workloads  # noqa: E402


def main(n_sample=256):
    d = workloads.workload("nacl32")
    pos, Q, L, n = d["pos"], d["Q"], d["L"], d["n_el"]
    idx = np.sort(np.random.default_rng(1234).choice(len(Q), n_sample, replace=False))
    pe, ge = ewald.ewald(pos, Q, L, targets=idx, want_grad=True)
    Fe = -Q[idx, None] * ge
    f = fep3m.forward(pos, Q, L, n, want_grad=True)
    dx, _, _ = fep3m.vjp(f, Q)
    rows = np.column_stack([idx, pe, Fe, f["phi"][idx], -dx[idx]])
    out = os.path.join(HERE, "nacl32_sample.txt")
    with open(out, "w") as fh:
        fh.write("# jittered rock salt 32^3 (seed 2, jitter 1e-3 L), 32^3 mesh, q=1, n_sr=3\n")
        fh.write("# U_fep3m_oracle %.17g\n" % f["U"])
        fh.write("# columns: index phi_ewald Fx_ewald Fy_ewald Fz_ewald phi_fep3m Fx_fep3m Fy_fep3m Fz_fep3m\n")
        np.savetxt(fh, rows, fmt=["%d"] + ["%.17g"] * 8)
    print(out)


if __name__ == "__main__":
    main()
