"""Write the oracle's cross sections of the 32^3 down-sampled twin of the
128^3 precision workload.

Test infrastructure only: calls nothing but the oracle and the seeded input
generators.  The 128^3 prism (x = 40, m = 1.31 + 0.01i, aspect 1, +z
incidence, x-polarised) is too large for a CPU FP64 solve; its twin keeps the
voxel size in wavelengths (k dx = 2x/N = 0.625) on a 32^3 grid (x = 10).  The
oracle solves it with its FP64 FFT operator and the 3-level preconditioner
to a true relative residual of 1e-12 and evaluates C_ext, C_abs and C_sca
(C_sca by the FFT route).  Output: tests/golden/config3_twin32_oracle.txt.

    python -m oracle.twin_values
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from dda_inputs import prism_case  # noqa: E402
from oracle.problem import from_case  # noqa: E402


def main():
    case = prism_case(32, 10.0, 1.31 + 0.01j, 1.0)
    prob = from_case(case, 0)
    x, info = prob.solve_gmres("3", tol=1e-12, restart=100, maxiter=3000)
    res = np.linalg.norm(prob.rhs() - prob.matvec(x)) / np.linalg.norm(prob.rhs())
    cext, cabs, csca = prob.cross_sections(x)
    l, m, n = case.dims
    lines = ["# Oracle (CPU FP64) cross sections of the 32^3 twin of the 128^3 workload:",
             "# hexagonal prism N = 32, x = 10, m = 1.31 + 0.01i, aspect 1, +z incidence,",
             "# x-polarised; GMRES(100) with the 3-level preconditioner to a true relative",
             "# residual of 1e-12.  Written by oracle/twin_values.py.",
             "# l m n n_scatterer gmres_iters rel_resid",
             f"box {l} {m} {n} {int((case.mask() > 0).sum())} {info['iters']} {res:.3e}",
             f"c_ext {cext:.17e}", f"c_abs {cabs:.17e}", f"c_sca {csca:.17e}"]
    out = os.path.join(ROOT, "tests", "golden", "config3_twin32_oracle.txt")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
